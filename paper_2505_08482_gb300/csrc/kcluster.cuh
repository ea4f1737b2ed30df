// Cluster-resident time stepping of the k-space scheme (Sec. 2.1): one thread-block cluster
// of C CTAs per data set runs a whole range of time steps with the wavefield on chip.
//
// CTA j of the cluster owns grid rows [row0(j), row0(j+1)) and half-spectrum columns
// [col0(j), col0(j+1)).  The state (u_x, u_y, rho_x, rho_y) of its rows lives in its shared
// memory for the whole launch.  A step has the four phases of the launched passes:
//   column G  (FFT_y, i k kappa e^{+ik dx/2}, IFFT_y of the pressure's row spectra),
//   velocity rows (inverse row FFTs, PML update of u, row R2C of u),
//   column D  (the same with the D factors on the two velocity spectra),
//   density rows (inverse row FFTs, PML update of rho, p = c^2 (rho_x + rho_y), sensor gather,
//                 pressure history, checkpoints, row R2C of p).
// Between phases the data changes owner through distributed shared memory: a row phase
// stores each row's spectrum values into the column buffer of the CTA that owns the column,
// a column phase stores its results into the row buffer of the CTA that owns the row, and a
// cluster barrier (release / acquire) ends every phase.  A CTA uses its own row buffer as the
// scratch of its row transforms and its column buffer as the scratch of its column
// transforms: other CTAs write a row buffer only during column phases and a column buffer
// only during row phases, so one barrier per phase is all the ordering needed.  The control
// flow is the same in every CTA (no waits on flags; barrier counts are uniform), and global
// memory is touched only for the medium and tables at the start, the traces, the pressure
// history, the checkpoints and the final state.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>

#include "kfixed.cuh"

namespace pat {

__device__ __forceinline__ unsigned cluster_rank() {
    unsigned r;
    asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
    return r;
}
// all threads of every CTA of the cluster; orders shared::cluster (and global) accesses
__device__ __forceinline__ void cluster_sync() {
    asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}
// store v at the same shared-memory location as p (this CTA's) in CTA `rank` of the cluster
__device__ __forceinline__ void st_cluster(const float2* p, unsigned rank, float2 v) {
    const uint32_t la = static_cast<uint32_t>(__cvta_generic_to_shared(p));
    uint32_t ra;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(ra) : "r"(la), "r"(rank));
    asm volatile("st.shared::cluster.v2.f32 [%0], {%1, %2};" ::"r"(ra), "f"(v.x), "f"(v.y) : "memory");
}

// v, opaque to the optimiser: values derived from it inside a loop iteration are not hoisted
// out of the time loop (which would keep every phase's precomputed indices live at once)
__device__ __forceinline__ int opaque(int v) {
    asm volatile("" : "+r"(v));
    return v;
}

// B layout of the packed inverse from half-spectrum rows in shared memory (as load_c2r_b)
template <class F>
__device__ __forceinline__ void load_c2r_b_sh(float2 (&b)[F::BV], int k1, const float2* ra, const float2* rb) {
    static_for<0, F::BV>([&](auto I) {
        constexpr int k2 = decltype(I)::value;
        const int kx = k1 + F::BT * k2;
        float2 z;
        if (2 * kx <= F::N) {
            float2 a = ra[kx], bb = rb[kx];
            if (kx == 0 || 2 * kx == F::N) {
                a.y = 0.f;
                bb.y = 0.f;
            }
            z = make_float2(a.x - bb.y, a.y + bb.x);
        } else {
            const int kk = F::N - kx;
            const float2 a = ra[kk], bb = rb[kk];
            z = make_float2(a.x + bb.y, bb.x - a.y);
        }
        b[k2] = z;
    });
}

struct ClusterArgs {
    const float* cg;      // c on the grid [ninst][ng][ng]
    const float* p0;      // [K][n][n] (init)
    const float* state;   // restore: state [4][K][ng][ng] (u_x, u_y, rho_x, rho_y) at level n0
    float* state_out;     // state at level n1, or null
    float* y;             // traces [K][nt][m] (zeroed), or null
    float* hist;          // pressure history [K][s_eff][ng][ng] of levels >= hist_base, or null
    int hist_base;
    float* ckpt;          // checkpoints [slot][4][K][ng][ng] of levels j s (slot j - 1), or null
    int s;
    int n0, n1;           // start at level n0 and run the steps n0 .. n1 - 1
    int init;             // 1: level 0 from p0 (the first velocity update is the initial one)
    float sg, sd;         // scales of the G and D multipliers (normalisation folded in)
};

// NG: grid side, C: CTAs per cluster, rows on Fft2<RN1, RN2>, columns on Fft2<CN1, CN2>
template <int NG, int C, int RN1, int RN2, int CN1, int CN2>
struct ClusterImpl {
    using FR = Fft2<RN1, RN2>;
    using FC = Fft2<CN1, CN2>;
    static_assert(FR::N == NG && FC::N == NG, "one grid side");
    static constexpr int NG_ = NG, csize = C;
    static constexpr int HC = NG / 2 + 1;
    static constexpr int RMAX = (NG + C - 1) / C;
    static constexpr int CMAX = (HC + C - 1) / C;
    static constexpr int TR = FR::T, TC = FC::T;
    static constexpr int NTR = RMAX * TR, NTC = 2 * CMAX * TC;
    static constexpr int NT = ((NTR > NTC ? NTR : NTC) + 31) / 32 * 32;
    static constexpr int AV = FR::AV, AT = FR::AT;
    static constexpr int ZR = FR::ZS | 1;                      // odd row stride of the row scratch
    static constexpr int RB = (2 * RMAX * HC > RMAX * ZR) ? 2 * RMAX * HC : RMAX * ZR;   // float2
    static constexpr int CF = (NG > FC::ZS ? NG : FC::ZS) * CMAX;                       // float2 / field
    static constexpr int PN = NG + ((20 - NG % 32) % 32 + 32) % 32;   // row stride of P (= 20 mod 32)
    static constexpr int KH = NG / 2 + 1;   // kappa is even in ky: entries ky <= NG / 2
    // shared memory (bytes); the pressure rows P of the density phase share the row buffer
    static constexpr size_t o_rb = 0;
    static constexpr size_t o_cb = o_rb + size_t(RB) * sizeof(float2);
    static constexpr size_t o_tw = o_cb + size_t(2 * CF) * sizeof(float2);
    static constexpr size_t o_twA = o_tw + NG * sizeof(float2);
    static constexpr size_t o_twB = o_twA + NG * sizeof(float2);
    static constexpr size_t o_fy = o_twB + NG * sizeof(float2);
    static constexpr size_t o_fx = o_fy + NG * sizeof(float2);
    static constexpr size_t o_csq = o_fx + CMAX * sizeof(float2);
    static constexpr size_t o_kap = o_csq + size_t(RMAX) * NG * sizeof(float);
    static constexpr size_t o_ac = o_kap + size_t(CMAX) * KH * sizeof(float);
    static constexpr size_t o_as = o_ac + NG * sizeof(float);
    static constexpr size_t o_st = o_as + NG * sizeof(float);   // u_x, u_y, rho_x, rho_y rows [4][RMAX][NG]
    static constexpr size_t smem = o_st + size_t(4 * RMAX) * NG * sizeof(float);
    static_assert(size_t(RMAX) * PN * sizeof(float) <= size_t(RB) * sizeof(float2), "P fits the row buffer");
    static_assert(smem <= 232448, "one CTA's shared memory");

    static __device__ __forceinline__ int row0(int j) { return (j * NG) / C; }
    static __device__ __forceinline__ int col0(int j) { return (j * HC) / C; }
    static __device__ __forceinline__ int row_owner(int y) { return ((y + 1) * C - 1) / NG; }
    static __device__ __forceinline__ int col_owner(int kx) { return ((kx + 1) * C - 1) / HC; }

    // shared-memory regions (offsets from the dynamic shared base)
    static __device__ __forceinline__ unsigned char* smbase() {
        extern __shared__ __align__(16) unsigned char smraw[];
        return smraw;
    }
    static __device__ __forceinline__ float2* s_rb() { return reinterpret_cast<float2*>(smbase() + o_rb); }
    static __device__ __forceinline__ float2* s_cb() { return reinterpret_cast<float2*>(smbase() + o_cb); }
    static __device__ __forceinline__ float2* s_tw() { return reinterpret_cast<float2*>(smbase() + o_tw); }
    static __device__ __forceinline__ float2* s_twA() { return reinterpret_cast<float2*>(smbase() + o_twA); }
    static __device__ __forceinline__ float2* s_twB() { return reinterpret_cast<float2*>(smbase() + o_twB); }
    static __device__ __forceinline__ float2* s_fy() { return reinterpret_cast<float2*>(smbase() + o_fy); }
    static __device__ __forceinline__ float2* s_fx() { return reinterpret_cast<float2*>(smbase() + o_fx); }
    static __device__ __forceinline__ float* s_P() { return reinterpret_cast<float*>(smbase() + o_rb); }
    static __device__ __forceinline__ float* s_csq() { return reinterpret_cast<float*>(smbase() + o_csq); }
    static __device__ __forceinline__ float* s_kap() { return reinterpret_cast<float*>(smbase() + o_kap); }
    static __device__ __forceinline__ float* s_ac() { return reinterpret_cast<float*>(smbase() + o_ac); }
    static __device__ __forceinline__ float* s_as() { return reinterpret_cast<float*>(smbase() + o_as); }
    static __device__ __forceinline__ float* s_st() { return reinterpret_cast<float*>(smbase() + o_st); }

    // Column phase: mode 0 (G): field 0 -> (MX, MY) x it into fields 0, 1 of the row buffers;
    // mode 1 (D): fields 0, 1 -> (MX f0, MY f1).  op: 0 G factors, 1 D factors.
    static __device__ __noinline__ void col_phase(int mode, int op, float scale, int kx0, int nc) {
        const int tid = opaque(int(threadIdx.x));
        kx0 = opaque(kx0);
        const int f = tid / (CMAX * TC), tl = tid - f * (CMAX * TC);
        const int c = tl % CMAX, idx = tl / CMAX;
        const bool colt = f < 2;
        const bool own_fwd = mode != 0 || f == 0;
        float2* Zf = s_cb() + (colt ? f : 0) * CF + c;
        float2 a[FC::AV];
        if (colt && own_fwd && idx < FC::AT)
            static_for<0, FC::AV>([&](auto I) {
                constexpr int n1 = decltype(I)::value;
                a[n1] = Zf[(FC::AT * n1 + idx) * CMAX];
            });
        __syncthreads();
        if (colt && own_fwd && idx < FC::AT) FC::template fwd_a<CMAX>(a, idx, Zf, s_tw());
        __syncthreads();
        float2 b[FC::BV];
        const bool bact = colt && idx < FC::BT;
        if (bact) {
            FC::template fwd_b_load<CMAX>(b, idx, own_fwd ? Zf : s_cb() + c);
            FC::fwd_b(b);
            const float2 mx0 = s_fx()[c];
            static_for<0, FC::BV>([&](auto I) {
                constexpr int k2 = decltype(I)::value;
                const int ky = idx + FC::BT * k2;
                float2 m = (f == 0) ? mx0 : s_fy()[ky];
                if (op == 1) m.x = -m.x;   // D factor = -conj(G factor)
                b[k2] = cmul(b[k2], cscale(m, scale * s_kap()[c * KH + (ky <= NG / 2 ? ky : NG - ky)]));
            });
        }
        __syncthreads();   // every read of the forward stage done before the inverse overwrites it
        if (bact) FC::template inv_b<CMAX>(b, idx, Zf, s_tw());
        __syncthreads();
        if (colt && idx < FC::AT && c < nc) {
            FC::template inv_a_load<CMAX>(a, idx, Zf);
            FC::inv_a(a);
            const int kx = kx0 + c;
            static_for<0, FC::AV>([&](auto I) {
                constexpr int n1 = decltype(I)::value;
                const int yv = idx + FC::AT * n1;
                const int own = row_owner(yv);
                st_cluster(s_rb() + (f * RMAX + (yv - row0(own))) * HC + kx, unsigned(own), a[n1]);
            });
        }
    }

    // inverse row transform of the two packed input spectra (row buffer fields 0 and 1) of row r:
    // g.x, g.y of the two fields at x = ridx + AT n1 (A layout) in av.  Two barriers.
    static __device__ __forceinline__ void row_inverse(int r, int ridx, bool rowt, float2 (&av)[AV]) {
        float2 b[FR::BV];
        const bool bact = rowt && ridx < FR::BT;
        if (bact) load_c2r_b_sh<FR>(b, ridx, s_rb() + r * HC, s_rb() + (RMAX + r) * HC);
        __syncthreads();
        if (bact) FR::inv_b_t(b, ridx, s_rb() + r * ZR, s_twB());
        __syncthreads();
        if (rowt && ridx < AT) {
            FR::inv_a_load(av, ridx, s_rb() + r * ZR);
            FR::inv_a(av);
        }
        __syncthreads();   // the scratch is free again
    }

    // first step of the forward row transform of sequence q (A layout values in av) into its scratch row
    static __device__ __forceinline__ void row_forward_a(int q, int ridx, bool act, float2 (&av)[AV]) {
        if (act && ridx < AT) FR::fwd_a_t(av, ridx, s_rb() + q * ZR, s_twA());
    }
    // rest of the forward row transforms of nseq sequences and the split into half spectra:
    // sequence q's real part -> row ya(q) of field fa, imaginary part -> row yb(q) of field fb
    // (pairs: rows y0 + 2q and y0 + 2q + 1 of field 0, the second only when below y0 + nr; else
    // row y0 + q of fields 0 and 1), stored into the owners' column buffers
    static __device__ __noinline__ void row_finish_scatter(int y0, int nr, bool pairs) {
        const int t = threadIdx.x;
        const int q = t / TR, ridx = t - q * TR;
        const int nseq = pairs ? (nr + 1) / 2 : nr;
        finish_fwd<FR>(s_rb() + q * ZR, ridx, q < nseq && ridx < FR::BT);
        const int fb = pairs ? 0 : 1;
        for (int i = t; i < nseq * HC; i += NT) {
            const int jj = i / HC, kx = i - jj * HC;
            const float2* W = s_rb() + jj * ZR;
            const float2 zk = W[kx];
            const float2 zm = W[kx == 0 ? 0 : NG - kx];
            const int own = col_owner(kx);
            const float2* dst = s_cb() + (kx - col0(own));
            const int ya = pairs ? y0 + 2 * jj : y0 + jj;
            const int yb = pairs ? (2 * jj + 1 < nr ? ya + 1 : -1) : ya;
            st_cluster(dst + ya * CMAX, unsigned(own), make_float2(0.5f * (zk.x + zm.x), 0.5f * (zk.y - zm.y)));
            if (yb >= 0)
                st_cluster(dst + fb * CF + yb * CMAX, unsigned(own),
                           make_float2(0.5f * (zk.y + zm.y), -0.5f * (zk.x - zm.x)));
        }
    }

    // sensor entries of the CTA's rows (CSR by grid row) and the traces of one level
    struct Sens {
        const int* srow;
        const int2* sent;
        const float4* sentw;
        float* ylv;   // y[k][lv][.], or null
    };

    // sensors of one level from the pressure rows P, then (scatter) the first step of the row R2C
    // of p, two rows per complex transform (P shares the row buffer with the transform scratch)
    static __device__ __noinline__ void p_sensors_pairs(const Sens& se_, int y0, int nr, bool scatter) {
        const int t = threadIdx.x;
        const int r = t / TR, ridx = t - r * TR;
        const float* P = s_P();
        if (se_.ylv) {
            const int e0 = se_.srow[y0], e1 = se_.srow[y0 + nr];
            for (int e = e0 + t; e < e1; e += NT) {
                const int2 se = se_.sent[e];
                const float4 sw = se_.sentw[e];
                const int rr = int(sw.w) - y0;
                const float v = sw.z * (sw.x * P[rr * PN + se.y] + sw.y * P[rr * PN + se.y + 1]);
                atomicAdd(se_.ylv + se.x, v);
            }
        }
        const int npair = (nr + 1) / 2;
        float2 av[AV];
        const bool act = scatter && r < npair;
        if (act && ridx < AT)
            static_for<0, AV>([&](auto I) {
                constexpr int n1 = decltype(I)::value;
                const int x = AT * n1 + ridx;
                av[n1] = make_float2(P[(2 * r) * PN + x], (2 * r + 1 < nr) ? P[(2 * r + 1) * PN + x] : 0.f);
            });
        __syncthreads();
        row_forward_a(r, ridx, act, av);
    }

    // The phases of a step, cut where everything a phase hands on is in shared memory, run as the
    // cases of one switch over the sub-phase index, each outlined (its own register allocation:
    // inlined into one time loop, the allocations of the phases overlap and spill).
    // velocity rows, first part: inverse row FFTs, u <- a'(a' u - g) (init: u = g / 2 first),
    // first step of the R2C of u
    static __device__ __noinline__ void phase_u(int y0, int nr, int init_u) {
        const int t = threadIdx.x;
        const int r = t / TR, ridx = t - r * TR;
        const bool rowt = r < nr, aact = rowt && ridx < AT;
        const int yy = y0 + min(r, nr - 1);
        float* uxs = s_st() + r * NG;
        float* uys = s_st() + (RMAX + r) * NG;
        float2 av[AV];
        row_inverse(r, ridx, rowt, av);
        if (aact) {
            const float ay = s_as()[yy];
            static_for<0, AV>([&](auto I) {
                constexpr int n1 = decltype(I)::value;
                const int x = ridx + AT * n1;
                const float ax = s_as()[x];
                const float2 gv = av[n1];
                const float uxo = init_u ? 0.5f * gv.x : uxs[x];
                const float uyo = init_u ? 0.5f * gv.y : uys[x];
                const float uxn = ax * (ax * uxo - gv.x);
                const float uyn = ay * (ay * uyo - gv.y);
                uxs[x] = uxn;
                uys[x] = uyn;
                av[n1] = make_float2(uxn, uyn);
            });
        }
        row_forward_a(r, ridx, rowt, av);
    }
    // density rows, first part: inverse row FFTs, rho <- a(a rho - g), p = c^2 (rho_x + rho_y)
    // into P and the history row hr (or null), the state into the checkpoint rows ck (or null,
    // f4 apart)
    static __device__ __noinline__ void phase_rho(int y0, int nr, float* hr, float* ck, size_t f4) {
        const int t = threadIdx.x;
        const int r = t / TR, ridx = t - r * TR;
        const bool rowt = r < nr, aact = rowt && ridx < AT;
        const int yy = y0 + min(r, nr - 1);
        float* rxs = s_st() + (2 * RMAX + r) * NG;
        float* rys = s_st() + (3 * RMAX + r) * NG;
        float2 av[AV];
        row_inverse(r, ridx, rowt, av);
        if (aact) {
            const float acy = s_ac()[yy];
            float* P = s_P() + r * PN;
            const float* csq = s_csq() + r * NG;
            const float* uxs = s_st() + r * NG;
            const float* uys = s_st() + (RMAX + r) * NG;
            if (hr) hr += size_t(yy) * NG;
            if (ck) ck += size_t(yy) * NG;
            static_for<0, AV>([&](auto I) {
                constexpr int n1 = decltype(I)::value;
                const int x = ridx + AT * n1;
                const float acx = s_ac()[x];
                const float2 gv = av[n1];
                const float rxn = acx * (acx * rxs[x] - gv.x);
                const float ryn = acy * (acy * rys[x] - gv.y);
                rxs[x] = rxn;
                rys[x] = ryn;
                const float pv = csq[x] * (rxn + ryn);
                P[x] = pv;
                if (hr) hr[x] = pv;
                if (ck) {
                    ck[x] = uxs[x];
                    ck[f4 + x] = uys[x];
                    ck[2 * f4 + x] = rxn;
                    ck[3 * f4 + x] = ryn;
                }
            });
        }
    }

    // per-CTA constants of the time loop, kept in shared memory: each phase reads what it needs
    // after the barrier that precedes it, so nothing is held in registers across the loop
    struct StepConst {
        float *hist, *ckpt, *y, *state_out;
        const int* srow;
        const int2* sent;
        const float4* sentw;
        size_t f4;
        int hist_base, s, s_eff, nt, m, n1, init, k, y0, nr, kx0, nc;
        float sg, sd;
    };

    // tables, initial state (p0 or a restored state) and the first row R2C; ends with every
    // CTA's column buffer complete
    static __device__ __noinline__ void setup(const Geo& g, const ClusterArgs& a, StepConst* sc) {
        const int tid = threadIdx.x;
        const int j = int(cluster_rank());
        const int k = blockIdx.y;
        const int y0 = row0(j), nr = row0(j + 1) - y0;
        const int kx0 = col0(j), nc = col0(j + 1) - kx0;
        if (tid == 0) {
            *sc = StepConst{a.hist, a.ckpt, a.y, a.state_out, g.srow, g.sent, g.sentw, size_t(g.K) * NG * NG,
                            a.hist_base, a.s, g.s_eff, g.nt, g.m, a.n1, a.init, k, y0, nr, kx0, nc, a.sg, a.sd};
        }
        for (int i = tid; i < NG; i += NT) {
            s_tw()[i] = g.tw[i];
            s_fy()[i] = g.fy[i];
            s_ac()[i] = g.a_cell[i];
            s_as()[i] = g.a_stag[i];
        }
        FR::fill_tables(s_twA(), s_twB(), g.tw, tid, NT);
        if (tid < CMAX) s_fx()[tid] = g.fx[min(kx0 + tid, HC - 1)];
        for (int i = tid; i < CMAX * KH; i += NT) {
            const int c = i / KH, ky = i - c * KH;
            s_kap()[i] = g.kappa_t[size_t(min(kx0 + c, HC - 1)) * NG + ky];
        }
        const float* cgk = medium_of(g, a.cg, k) + size_t(y0) * NG;
        for (int i = tid; i < nr * NG; i += NT) {
            const float v = cgk[i];
            s_csq()[i] = v * v;
        }
        // row threads: row r of the CTA, cells x = ridx + AT n1
        const int r = tid / TR, ridx = tid - r * TR;
        const bool aact = r < nr && ridx < AT;
        const int yy = y0 + min(r, nr - 1);
        const size_t f4 = size_t(g.K) * NG * NG;
        const size_t rowo = (size_t(k) * NG + yy) * NG;
        float* uxs = s_st() + r * NG;
        float* uys = s_st() + (RMAX + r) * NG;
        float* rxs = s_st() + (2 * RMAX + r) * NG;
        float* rys = s_st() + (3 * RMAX + r) * NG;
        // every CTA of the cluster has started (its shared memory may be written) and the tables are in
        cluster_sync();
        if (aact) {
            const int yd = yy - g.P;
            float* hr = (a.hist && a.n0 >= a.hist_base)
                            ? a.hist + (size_t(k) * g.s_eff + (a.n0 - a.hist_base)) * NG * NG + size_t(yy) * NG
                            : nullptr;
            static_for<0, AV>([&](auto I) {
                constexpr int n1 = decltype(I)::value;
                const int x = ridx + AT * n1;
                const float c2 = s_csq()[r * NG + x];
                float pv;
                if (a.init) {
                    const int xd = x - g.P;
                    pv = (xd >= 0 && xd < g.n && yd >= 0 && yd < g.n) ? a.p0[(size_t(k) * g.n + yd) * g.n + xd] : 0.f;
                    uxs[x] = 0.f;
                    uys[x] = 0.f;
                    rxs[x] = pv / (2.f * c2);
                    rys[x] = rxs[x];
                } else {
                    uxs[x] = a.state[rowo + x];
                    uys[x] = a.state[f4 + rowo + x];
                    const float r0 = a.state[2 * f4 + rowo + x], r1 = a.state[3 * f4 + rowo + x];
                    rxs[x] = r0;
                    rys[x] = r1;
                    pv = c2 * (r0 + r1);
                }
                s_P()[r * PN + x] = pv;
                if (hr) hr[x] = pv;
            });
        }
        __syncthreads();
        Sens se{g.srow, g.sent, g.sentw, a.y ? a.y + (size_t(k) * g.nt + a.n0) * g.m : nullptr};
        p_sensors_pairs(se, y0, nr, a.n1 > a.n0);
        __syncthreads();
        if (a.n1 > a.n0) row_finish_scatter(y0, nr, true);
        cluster_sync();
    }

    // the state of the CTA's rows into state_out
    static __device__ __noinline__ void finish(const StepConst* sc) {
        const int tid = threadIdx.x;
        const int r = tid / TR, ridx = tid - r * TR;
        if (!sc->state_out || r >= sc->nr || ridx >= AT) return;
        const size_t f4 = sc->f4;
        const size_t rowo = (size_t(sc->k) * NG + sc->y0 + r) * NG;
        float* out = sc->state_out + rowo;
        static_for<0, AV>([&](auto I) {
            constexpr int n1 = decltype(I)::value;
            const int x = ridx + AT * n1;
            static_for<0, 4>([&](auto F) {
                constexpr int fi = decltype(F)::value;
                out[fi * f4 + x] = s_st()[(fi * RMAX + r) * NG + x];
            });
        });
    }

    static __device__ __forceinline__ void forward(const Geo& g, const ClusterArgs& a) {
        __shared__ StepConst sc;
        setup(g, a, &sc);
        // sub-phases of a step: 0 column G | 1 velocity rows | 2 their R2C scatter | 3 column D |
        // 4 density rows | 5 sensors and the first R2C step of p | 6 its scatter; a cluster
        // barrier ends 0, 2, 3 and 6, a CTA barrier the others
        for (int q = 7 * a.n0; q < 7 * a.n1; ++q) {
            const int n = q / 7, sub = q - 7 * n;
            const int lv = n + 1;
            switch (sub) {
                case 0:
                    col_phase(0, 0, sc.sg, sc.kx0, sc.nc);
                    break;
                case 1:
                    phase_u(sc.y0, sc.nr, sc.init && n == 0);
                    break;
                case 2:
                    row_finish_scatter(sc.y0, sc.nr, false);
                    break;
                case 3:
                    col_phase(1, 1, sc.sd, sc.kx0, sc.nc);
                    break;
                case 4: {
                    const int k = sc.k;
                    float* hr = (sc.hist && lv >= sc.hist_base)
                                    ? sc.hist + (size_t(k) * sc.s_eff + (lv - sc.hist_base)) * NG * NG
                                    : nullptr;
                    float* ck = (sc.ckpt && lv % sc.s == 0)
                                    ? sc.ckpt + size_t(lv / sc.s - 1) * 4 * sc.f4 + size_t(k) * NG * NG
                                    : nullptr;
                    phase_rho(sc.y0, sc.nr, hr, ck, sc.f4);
                    break;
                }
                case 5: {
                    Sens se{sc.srow, sc.sent, sc.sentw, sc.y ? sc.y + (size_t(sc.k) * sc.nt + lv) * sc.m : nullptr};
                    p_sensors_pairs(se, sc.y0, sc.nr, lv < sc.n1);
                    break;
                }
                default:
                    if (lv < sc.n1) row_finish_scatter(sc.y0, sc.nr, true);
            }
            if (sub == 0 || sub == 2 || sub == 3 || sub == 6)
                cluster_sync();
            else
                __syncthreads();
        }
        finish(&sc);
    }
};

template <class CI>
__global__ void __launch_bounds__(CI::NT, 1) kc_forward(Geo g, ClusterArgs a) {
    CI::forward(g, a);
}

// launch table of the cluster-resident sweep of one grid side
struct ClusterOps {
    int ng, csize;
    int (*configure)();
    int (*forward)(const Geo&, cudaStream_t, const ClusterArgs&);
    int (*capacity)();   // clusters the current GPU runs at once (0: none)
};

template <class CI>
struct ClusterLaunch {
    static int configure() {
        cudaError_t e = cudaFuncSetAttribute((const void*)kc_forward<CI>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             int(CI::smem));
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute((const void*)kc_forward<CI>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
        return e == cudaSuccess ? PAT_OK : cuda_fail(e, "cudaFuncSetAttribute(kc_forward)");
    }
    static int forward(const Geo& g, cudaStream_t st, const ClusterArgs& a) {
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3(CI::csize, g.K);
        cfg.blockDim = dim3(CI::NT);
        cfg.dynamicSmemBytes = CI::smem;
        cfg.stream = st;
        cudaLaunchAttribute attr[1];
        attr[0].id = cudaLaunchAttributeClusterDimension;
        attr[0].val.clusterDim.x = CI::csize;
        attr[0].val.clusterDim.y = 1;
        attr[0].val.clusterDim.z = 1;
        cfg.attrs = attr;
        cfg.numAttrs = 1;
        cudaError_t e = cudaLaunchKernelEx(&cfg, kc_forward<CI>, g, a);
        if (e != cudaSuccess) {
            cudaFuncAttributes fa{};
            cudaFuncGetAttributes(&fa, (const void*)kc_forward<CI>);
            int ncl = -1;
            cfg.gridDim = dim3(CI::csize, 1);
            cudaOccupancyMaxActiveClusters(&ncl, (const void*)kc_forward<CI>, &cfg);
            set_error("cudaLaunchKernelEx(kc_forward): %s (%d registers, %d max threads, %zu B local, %zu B shared, "
                      "%d clusters fit)", cudaGetErrorString(e), fa.numRegs, fa.maxThreadsPerBlock,
                      size_t(fa.localSizeBytes), CI::smem, ncl);
            return PAT_ECUDA;
        }
        return PAT_OK;
    }
    static int capacity() {
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3(CI::csize, 1);
        cfg.blockDim = dim3(CI::NT);
        cfg.dynamicSmemBytes = CI::smem;
        cudaLaunchAttribute attr[1];
        attr[0].id = cudaLaunchAttributeClusterDimension;
        attr[0].val.clusterDim.x = CI::csize;
        attr[0].val.clusterDim.y = 1;
        attr[0].val.clusterDim.z = 1;
        cfg.attrs = attr;
        cfg.numAttrs = 1;
        int n = 0;
        return cudaOccupancyMaxActiveClusters(&n, (const void*)kc_forward<CI>, &cfg) == cudaSuccess ? n : 0;
    }
    static ClusterOps ops() { return ClusterOps{CI::NG_, CI::csize, &configure, &forward, &capacity}; }
};

const ClusterOps* cluster_ops_for(int ng);   // nullptr if the side has no cluster-resident sweep

}  // namespace pat

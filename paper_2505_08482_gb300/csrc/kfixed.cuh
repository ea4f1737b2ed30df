// Fixed-size passes of the k-space scheme for grid sides Ng = N1 * N2 known at
// compile time, built on the two-level register FFT of fft2l.cuh.
//
// Column pass (one launch = FFT_y, k-space multiply, IFFT_y of CC spectral
// columns per CTA): global -> registers (A layout) -> DFT_N1 -> transpose ->
// DFT_N2 -> multiply by i k kappa e^{+-i k dx/2} -> inverse DFT_N2 ->
// transpose -> inverse DFT_N1 -> global: two shared-memory transposes in all.
//
// Row passes (RR grid rows per CTA): the packed half spectra are read straight
// into the B layout, inverse-transformed through one transpose into the A
// layout, where each thread holds the real-space values of its row at
// x = n2 + N2 n1 and applies the pointwise update (PML, equation of state,
// adjoint terms); the forward transform of the updated fields goes back
// through one transpose and a last shared-memory pass splits the two packed
// half spectra.  Results are the same as the generic Stockham passes.
//
// The pointwise update needs the CTA's rows of the state, the medium and the
// PML factors.  They are fetched before the programmatic-dependency wait so that
// their latency overlaps the preceding kernel and the inverse transform: into
// registers (STAGE = false) or, with STAGE = true, by TMA bulk copies into
// shared memory (the RR rows of a data set are contiguous: one copy per array),
// which leaves the registers to the FFT so that more CTAs share an SM.
//
// In shared memory the row passes keep their twiddles in two per-layout tables (the threads of
// one transform step read consecutive entries) and pad the row strides of their transpose
// buffers and real rows (RowPad), so that rows sharing a warp fall on different banks.
//
// The same pass bodies also run inside the persistent forward sweep (PersistentImpl at the end
// of this file), which takes their tiles from a work queue instead of a launch grid.
#pragma once

#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>
#include <type_traits>

#include "dcheck.cuh"
#include "fft2l.cuh"
#include "geo.cuh"
#include "sync.cuh"

namespace pat {

// ---------------------------------------------------------------------------
// launch table of one fixed size / tile variant
struct FixedOps {
    int ng, rr, cc;
    int (*configure)();
    void (*col)(const Geo&, cudaStream_t, float2*, float2*, int mode, int op, float scale);
    void (*row_u)(const Geo&, cudaStream_t, float2*, float2*, float*, float*, int kind, int init);
    void (*row_rho)(const Geo&, cudaStream_t, float2*, const float2*, float*, float*, const float*, int mode,
                    const float* p0, float* y, int tstep, float* hist, int hist_slot);
    void (*row_adj_rho)(const Geo&, cudaStream_t, float2*, float2*, float*, float*, float*, const float*,
                        int first, const float* resid, int tstep, const float* hist, int hist_slot);
    // column pass for passes that run alone on the GPU (nullptr: col)
    void (*col_solo)(const Geo&, cudaStream_t, float2*, float2*, int mode, int op, float scale);
    // row passes of the segment recompute, which shares the GPU with the adjoint (nullptr: row_u, row_rho)
    void (*row_u_rc)(const Geo&, cudaStream_t, float2*, float2*, float*, float*, int kind, int init);
    void (*row_rho_rc)(const Geo&, cudaStream_t, float2*, const float2*, float*, float*, const float*, int mode,
                       const float* p0, float* y, int tstep, float* hist, int hist_slot);
};

const FixedOps* fixed_ops_for(int ng, int variant);   // nullptr if no fixed size matches
int fixed_variants(int ng);                           // number of tile variants for ng (0 if none)

// L2 load of a spectrum element (written by other CTAs of the preceding kernel)
__device__ __forceinline__ float2 ld_spec(const float2* p) { return __ldcg(p); }

// ---------------------------------------------------------------------------
// Where a pass body runs.  A body computes one tile (bx) of one data set (k) and has two
// dependency points: state_ready() before it fetches the state rows that the pass two
// passes back wrote, input_ready() before it reads the spectra that the preceding pass
// wrote.  A launched pass (one tile per CTA) relies on stream order for the first and
// waits for the preceding kernel (programmatic dependent launch) at the second.  The
// forward row passes can also copy the state rows they write into a checkpoint (ck_*);
// a launched pass has no checkpoint target.
struct LaunchedCtx {
    int bx, k;
    // state rows written by earlier kernels of the stream: ordinary loads
    __device__ __forceinline__ float ld(const float* p) const { return *p; }
    __device__ __forceinline__ void state_ready() const {}
    __device__ __forceinline__ void input_ready() const { pdl_wait_then_release(); }
    __device__ __forceinline__ float* ck_a() const { return nullptr; }
    __device__ __forceinline__ float* ck_b() const { return nullptr; }
};

// ---------------------------------------------------------------------------
// B layout of the packed inverse: b[k2] = Z[k1 + N1 k2] where Z is the full
// spectrum of a + i b built from the half spectra rows ra (of a) and rb (of b).
template <class F>
__device__ __forceinline__ void load_c2r_b(float2 (&b)[F::N2], int k1, const float2* __restrict__ ra,
                                           const float2* __restrict__ rb) {
    static_for<0, F::N2>([&](auto I) {
        constexpr int k2 = decltype(I)::value;
        const int kx = k1 + F::N1 * k2;
        float2 z;
        if (2 * kx <= F::N) {
            float2 a = ld_spec(ra + kx), bb = ld_spec(rb + kx);
            if (kx == 0 || 2 * kx == F::N) {
                a.y = 0.f;
                bb.y = 0.f;
            }
            z = make_float2(a.x - bb.y, a.y + bb.x);
        } else {
            const int kk = F::N - kx;
            const float2 a = ld_spec(ra + kk), bb = ld_spec(rb + kk);
            z = make_float2(a.x + bb.y, bb.x - a.y);
        }
        b[k2] = z;
    });
}

__device__ __forceinline__ void col_mults(const Geo& g, int kx, int ky, int op, float scale, float2& mx,
                                          float2& my) {
    const float kap = scale * g.kappa_t[size_t(kx) * g.ng + ky];
    mx = g.fx[kx];
    my = g.fy[ky];
    if (op == 1) {  // D factor = -conj(G factor)
        mx.x = -mx.x;
        my.x = -my.x;
    }
    mx = cscale(mx, kap);
    my = cscale(my, kap);
}

// ---------------------------------------------------------------------------
// column pass; mode 0: A -> (MX A, MY A) into (A, B); 1: (A, B) -> (MX A, MY B); 2: MX A + MY B -> A.
// The two fields (or the two outputs) of a column are handled by separate threads (f = 0, 1);
// in mode 0 they share the first transform stage.
// Tables and twiddles are staged before the dependency wait, the columns read after it.
// LEAN = false: the multipliers MX, MY of the CTA's columns are tabulated in shared memory before
// the dependency wait (off the critical path of a chain of passes); LEAN = true: they are formed
// where they are used from the factors and kappa (less shared memory and fewer instructions, so
// more CTAs per SM and a higher rate when a launch has many waves, at the cost of a longer
// critical path after the wait).
template <int N1, int N2, int CC, bool LEAN = false>
struct ColSmem {
    using F = Fft2<N1, N2>;
    static constexpr int tables = LEAN ? 2 * F::N + CC + (F::N * CC + 1) / 2 : F::N + 2 * F::N * CC;   // float2
    static constexpr size_t bytes = (size_t(tables) + 4 * F::ZS * CC) * sizeof(float2);
};

template <int N1, int N2, int CC, class Ctx, bool LEAN = false>
__device__ __forceinline__ void col_body(const Geo& g, const Ctx& ctx, float2* __restrict__ A,
                                         float2* __restrict__ B, int mode, int op, float scale) {
    using F = Fft2<N1, N2>;
    ctx.state_ready();
    constexpr int N = F::N;
    constexpr int NT = 2 * CC * F::T;
    extern __shared__ float2 sm[];
    float2* tw = sm;                        // [N]
    // LEAN: y factor of the pass's operator [N], x factors of the CTA's columns [CC], scale * kappa
    // at (ky, c) [N][CC] (floats); else MX, MY at (ky, c) [N][CC] each
    float2* FY = tw + N;
    float2* FXC = FY + N;
    float* KP = reinterpret_cast<float*>(FXC + CC);
    float2* MX = tw + N;
    float2* MY = MX + N * CC;
    float2* Zf = sm + ColSmem<N1, N2, CC, LEAN>::tables;   // forward transposes of the two threads' fields, [2][ZS][CC]
    float2* Zi = Zf + 2 * F::ZS * CC;       // inverse transposes of the two outputs, [2][ZS][CC]
    const int k = ctx.k;
    const int f = threadIdx.x / (CC * F::T);
    const int tl = threadIdx.x - f * (CC * F::T);
    const int c = tl % CC, idx = tl / CC;
    const int kx = ctx.bx * CC + c;
    const bool colok = kx < g.hc;
    const int kxc = colok ? kx : g.hc - 1;
    const size_t base = size_t(k) * N * g.hp + kxc;
    if constexpr (LEAN) {
        // MX = fx(kx) kap, MY = fy(ky) kap (kap = scale kappa(kx, ky); D: -conj of the G factors)
        // are formed where they are used, from the factors and kappa staged here
        static_for<0, (N + NT - 1) / NT>([&](auto I) {
            const int i = decltype(I)::value * NT + threadIdx.x;
            if (i < N) {
                tw[i] = g.tw[i];
                float2 v = g.fy[i];
                if (op == 1) v.x = -v.x;
                FY[i] = v;
            }
        });
        if (threadIdx.x < CC) {
            float2 v = g.fx[min(ctx.bx * CC + int(threadIdx.x), g.hc - 1)];
            if (op == 1) v.x = -v.x;
            FXC[threadIdx.x] = v;
        }
        static_for<0, (N * CC + NT - 1) / NT>([&](auto I) {
            const int i = decltype(I)::value * NT + threadIdx.x;
            if (i < N * CC) {
                const int cc = i / N, ky = i - cc * N;
                const int kxs = min(ctx.bx * CC + cc, g.hc - 1);
                KP[ky * CC + cc] = scale * g.kappa_t[size_t(kxs) * g.ng + ky];
            }
        });
    } else {
        static_for<0, (N + NT - 1) / NT>([&](auto I) {
            const int i = decltype(I)::value * NT + threadIdx.x;
            if (i < N) tw[i] = g.tw[i];
        });
        static_for<0, (N * CC + NT - 1) / NT>([&](auto I) {
            const int i = decltype(I)::value * NT + threadIdx.x;
            if (i < N * CC) {
                const int cc = i % CC, ky = i / CC;
                const int kxs = min(ctx.bx * CC + cc, g.hc - 1);
                float2 mx, my;
                col_mults(g, kxs, ky, op, scale, mx, my);
                MX[i] = mx;
                MY[i] = my;
            }
        });
    }
    ctx.input_ready();
    float2* Zmine = Zf + f * F::ZS * CC + c;
    // mode 0 has one input: the f = 1 threads read the f = 0 threads' first transform stage
    const bool own_fwd = mode != 0 || f == 0;
    float2 a[N1];
    if (idx < N2 && own_fwd) {
        const float2* src = (mode == 0 || f == 0) ? A : B;
        static_for<0, N1>([&](auto I) {
            constexpr int n1 = decltype(I)::value;
            a[n1] = ld_spec(src + base + size_t(N2 * n1 + idx) * g.hp);
        });
    }
    __syncthreads();   // twiddles and multipliers staged by all threads
    if (idx < N2 && own_fwd) F::template fwd_a<CC>(a, idx, Zmine, tw);
    __syncthreads();
    float2 b[N2];
    if (idx < N1) {
        F::template fwd_b_load<CC>(b, idx, own_fwd ? Zmine : Zf + c);
        F::fwd_b(b);
        if constexpr (LEAN) {
            const float2 fxm = FXC[c];
            static_for<0, N2>([&](auto I) {
                constexpr int k2 = decltype(I)::value;
                const int ky = idx + N1 * k2;
                b[k2] = cmul(b[k2], cscale(f == 0 ? fxm : FY[ky], KP[ky * CC + c]));
            });
        } else {
            const float2* Mm = (f == 0) ? MX : MY;
            static_for<0, N2>([&](auto I) {
                constexpr int k2 = decltype(I)::value;
                b[k2] = cmul(b[k2], Mm[(idx + N1 * k2) * CC + c]);
            });
        }
        if (mode == 2 && f == 1) {   // hand the product to the f = 0 thread of the same column
            static_for<0, N2>([&](auto I) { Zi[((F::ZS + idx * N2 + decltype(I)::value) * CC) + c] = b[decltype(I)::value]; });
        }
    }
    if (mode == 2) __syncthreads();
    if (idx < N1 && (mode != 2 || f == 0)) {
        if (mode == 2)
            static_for<0, N2>([&](auto I) {
                b[decltype(I)::value] = cadd(b[decltype(I)::value], Zi[((F::ZS + idx * N2 + decltype(I)::value) * CC) + c]);
            });
        F::template inv_b<CC>(b, idx, Zi + f * F::ZS * CC + c, tw);
    }
    __syncthreads();
    if (idx < N2 && colok && (mode != 2 || f == 0)) {
        F::template inv_a_load<CC>(a, idx, Zi + f * F::ZS * CC + c);
        F::inv_a(a);
        float2* dst = f == 0 ? A : B;
        static_for<0, N1>([&](auto I) {
            constexpr int n1 = decltype(I)::value;
            dst[base + size_t(idx + N2 * n1) * g.hp] = a[n1];
        });
    }
}

template <int N1, int N2, int CC>
__global__ void __launch_bounds__(2 * CC * Fft2<N1, N2>::T) kf_col(Geo g, float2* __restrict__ A,
                                                                  float2* __restrict__ B, int mode, int op,
                                                                  float scale) {
    col_body<N1, N2, CC>(g, LaunchedCtx{int(blockIdx.x), int(blockIdx.y)}, A, B, mode, op, scale);
}

template <int N1, int N2, int CC>
__global__ void __launch_bounds__(2 * CC * Fft2<N1, N2>::T) kf_col_lean(Geo g, float2* __restrict__ A,
                                                                       float2* __restrict__ B, int mode, int op,
                                                                       float scale) {
    col_body<N1, N2, CC, LaunchedCtx, true>(g, LaunchedCtx{int(blockIdx.x), int(blockIdx.y)}, A, B, mode, op, scale);
}

// Column pass on the three-level transform (Fft3): the same modes and multipliers as col_body,
// with three times as many threads per column (every thread holds at most max(NA, NM, NB)
// values), so that a launch at K = 8 keeps about three times as many warps on each SM.
// Shared buffers per field: Z1 (A -> M forward, B -> M inverse), Z2 (M -> B forward, M -> A
// inverse); the f = 1 threads of mode 0 read the f = 0 threads' M -> B buffer.
template <int NA, int NM, int NB, int CC, class Ctx>
__device__ __forceinline__ void col3_body(const Geo& g, const Ctx& ctx, float2* __restrict__ A,
                                          float2* __restrict__ B, int mode, int op, float scale) {
    using F = Fft3<NA, NM, NB>;
    ctx.state_ready();
    constexpr int N = F::N, T = F::T, ZS = F::ZS;
    constexpr int NT = 2 * CC * T;
    extern __shared__ float2 sm[];
    float2* twA = sm;                       // [N]
    float2* twM = twA + N;                  // [N2]
    float2* MX = twM + F::N2;               // [N][CC] x multiplier at (ky, c)
    float2* MY = MX + N * CC;               // [N][CC]
    float2* Z1 = MY + N * CC;               // [2][ZS][CC]
    float2* Z2 = Z1 + 2 * ZS * CC;          // [2][ZS][CC]
    const int k = ctx.k;
    const int f = threadIdx.x / (CC * T);
    const int tl = threadIdx.x - f * (CC * T);
    const int c = tl % CC, idx = tl / CC;
    const int kx = ctx.bx * CC + c;
    const bool colok = kx < g.hc;
    const int kxc = colok ? kx : g.hc - 1;
    const size_t base = size_t(k) * N * g.hp + kxc;
    F::fill_tables(twA, twM, g.tw, threadIdx.x, NT);
    for (int i = threadIdx.x; i < N * CC; i += NT) {
        const int cc = i % CC, ky = i / CC;
        const int kxs = min(ctx.bx * CC + cc, g.hc - 1);
        float2 mx, my;
        col_mults(g, kxs, ky, op, scale, mx, my);
        MX[i] = mx;
        MY[i] = my;
    }
    ctx.input_ready();
    float2* Z1f = Z1 + f * ZS * CC + c;
    float2* Z2f = Z2 + f * ZS * CC + c;
    const bool own_fwd = mode != 0 || f == 0;
    float2 a[NA];
    if (idx < F::AT && own_fwd) {
        const float2* src = (mode == 0 || f == 0) ? A : B;
        static_for<0, NA>([&](auto I) {
            constexpr int n1 = decltype(I)::value;
            a[n1] = ld_spec(src + base + size_t(F::AT * n1 + idx) * g.hp);
        });
    }
    __syncthreads();   // twiddles and multipliers staged by all threads
    if (idx < F::AT && own_fwd) F::template fwd_a_t<CC>(a, idx, Z1f, twA);
    __syncthreads();
    if (idx < F::MT && own_fwd) F::template fwd_m<CC>(idx, Z1f, Z2f, twM);
    __syncthreads();
    float2 b[NB];
    const float2* Mm = (f == 0) ? MX : MY;
    float2* Zh = Z1 + ZS * CC + c;   // mode 2: the f = 1 product handed to the f = 0 thread
    if (idx < F::BT) {
        F::template fwd_b_load<CC>(b, idx, own_fwd ? Z2f : Z2 + c);
        F::fwd_b(b);
        static_for<0, NB>([&](auto I) {
            constexpr int k2 = decltype(I)::value;
            b[k2] = cmul(b[k2], Mm[(idx + F::BT * k2) * CC + c]);
        });
        if (mode == 2 && f == 1)
            static_for<0, NB>([&](auto I) { Zh[(idx * NB + decltype(I)::value) * CC] = b[decltype(I)::value]; });
    }
    if (mode == 2) __syncthreads();
    const bool inv = mode != 2 || f == 0;
    if (idx < F::BT && inv) {
        if (mode == 2)
            static_for<0, NB>([&](auto I) {
                b[decltype(I)::value] = cadd(b[decltype(I)::value], Zh[(idx * NB + decltype(I)::value) * CC]);
            });
        F::template inv_b_t<CC>(b, idx, Z1f, twM);
    }
    __syncthreads();
    if (idx < F::MT && inv) F::template inv_m<CC>(idx, Z1f, Z2f, twA);
    __syncthreads();
    if (idx < F::AT && colok && inv) {
        F::template inv_a_load<CC>(a, idx, Z2f);
        F::inv_a(a);
        float2* dst = f == 0 ? A : B;
        static_for<0, NA>([&](auto I) {
            constexpr int n1 = decltype(I)::value;
            dst[base + size_t(idx + F::AT * n1) * g.hp] = a[n1];
        });
    }
}

template <int NA, int NM, int NB, int CC>
__global__ void __launch_bounds__(2 * CC * Fft3<NA, NM, NB>::T) kf_col3(Geo g, float2* __restrict__ A,
                                                                       float2* __restrict__ B, int mode, int op,
                                                                       float scale) {
    col3_body<NA, NM, NB, CC>(g, LaunchedCtx{int(blockIdx.x), int(blockIdx.y)}, A, B, mode, op, scale);
}

// Split the natural-order spectra W[j] (of a_j + i b_j) of nseq rows into half spectra:
// a_j -> row rowa(j), b_j -> row rowb(j).
template <class F, int ZR, class RowA, class RowB>
__device__ __forceinline__ void unpack_rows(const float2* Z, int nseq, RowA rowa, RowB rowb) {
    constexpr int H = F::N / 2 + 1;
    for (int i = threadIdx.x; i < nseq * H; i += blockDim.x) {
        const int j = i / H, kx = i - j * H;
        const float2* W = Z + j * ZR;
        const float2 zk = W[kx];
        const float2 zm = W[kx == 0 ? 0 : F::N - kx];
        rowa(j)[kx] = make_float2(0.5f * (zk.x + zm.x), 0.5f * (zk.y - zm.y));
        rowb(j)[kx] = make_float2(0.5f * (zk.y + zm.y), -0.5f * (zk.x - zm.x));
    }
}

// finish the forward transforms whose A-layout halves fwd_a stored in Zs (nseq
// buffers of ZS): natural-order spectrum into Zs.  Contains two barriers.
template <class F>
__device__ __forceinline__ void finish_fwd(float2* Zs, int idx, bool active) {
    float2 b[F::N2];
    if (active) F::fwd_b_load(b, idx, Zs);
    __syncthreads();
    if (active) {
        F::fwd_b(b);
        static_for<0, F::N2>([&](auto I) { Zs[idx + F::N1 * decltype(I)::value] = b[decltype(I)::value]; });
    }
    __syncthreads();
}

// Row strides (elements) of the row passes' shared buffers: zs for a transpose buffer (float2),
// pn for a real row (float).  The unpadded strides (the Fft2 buffer size, the row length) put
// rows that share a warp on the same banks; these were chosen by counting the shared-memory
// wavefronts of the passes' main patterns (A- and B-layout steps, row stores, pair loads) for
// tiles of 4 and 8 rows, and never raise the count.
template <int N1, int N2>
struct RowPad {
    static constexpr int zs = Fft2<N1, N2>::ZS, pn = N1 * N2;
};
template <> struct RowPad<9, 12> { static constexpr int zs = 124, pn = 108; };
template <> struct RowPad<12, 9> { static constexpr int zs = 108, pn = 117; };
template <> struct RowPad<12, 12> { static constexpr int zs = 156, pn = 172; };
template <> struct RowPad<12, 15> { static constexpr int zs = 180, pn = 207; };
template <> struct RowPad<15, 12> { static constexpr int zs = 204, pn = 182; };
template <> struct RowPad<10, 20> { static constexpr int zs = 212, pn = 202; };
template <> struct RowPad<20, 10> { static constexpr int zs = 220, pn = 202; };
template <> struct RowPad<15, 20> { static constexpr int zs = 324, pn = 314; };
template <> struct RowPad<20, 15> { static constexpr int zs = 300, pn = 312; };

// Shared memory of the row passes: the two twiddle tables, two transpose buffers and RR real rows
// (base); staged: then ns arrays of RR rows, the PML factors, nc arrays of RR domain
// rows of width n, and the mbarrier.
template <class F, int RR>
struct RowSmem {
    static constexpr int ZR = RowPad<F::N1, F::N2>::zs, PN = RowPad<F::N1, F::N2>::pn;
    static_assert(ZR >= F::ZS && PN >= F::N, "padded strides");
    static constexpr size_t base = (2 * F::N + 2 * RR * ZR) * sizeof(float2) + RR * PN * sizeof(float);
    static constexpr size_t staged(int ns, int nc, int n) {
        return base + (size_t(ns) * RR + 1) * F::N * sizeof(float) + size_t(nc) * RR * n * sizeof(float) + 16;
    }
};

// bytes of nr consecutive rows of an Ng-wide field
template <int N>
__device__ __forceinline__ uint32_t rows_bytes(int nr) {
    return uint32_t(nr) * N * sizeof(float);
}

// ---------------------------------------------------------------------------
// velocity row pass; kind 0 forward: u <- a'(a' u - g) (init: u = g/2 first),
// kind 1 adjoint: t' = a'(ub + g), ub <- a' t'.  Then (A, B) <- R2C of the new pair.
// The state and PML factors are not written by the preceding kernel: fetched before the wait.
template <int N1, int N2, int RR, bool STAGE, bool LATE, class Ctx>
__device__ __forceinline__ void row_u_body(const Geo& g, const Ctx& ctx, float2* __restrict__ A,
                                           float2* __restrict__ B, float* __restrict__ ux, float* __restrict__ uy,
                                           int kind, int init) {
    using F = Fft2<N1, N2>;
    constexpr int N = F::N, T = F::T;
    constexpr int ZR = RowPad<N1, N2>::zs, PN = RowPad<N1, N2>::pn;   // padded row strides
    extern __shared__ float2 sm[];
    float2* twA = sm;       // twiddles of the A-layout step [N], read with consecutive n2 across threads
    float2* twB = sm + N;   // twiddles of the B-layout step [N], read with consecutive k1 across threads
    float2* Z0 = sm + 2 * N;
    float2* Z1 = Z0 + RR * ZR;
    float* Sx = reinterpret_cast<float*>(Z1 + RR * ZR) + RR * PN;   // staged u_x, u_y [RR][N] (after base)
    float* Sy = Sx + RR * N;
    float* Sa = Sy + RR * N;                                           // PML factors [N]
    uint64_t* mb = reinterpret_cast<uint64_t*>(Sa + N);
    const int k = ctx.k, y0 = ctx.bx * RR;
    const int r = threadIdx.x / T, idx = threadIdx.x % T;
    const int nr = min(RR, N - y0);
    const bool rowok = r < nr;
    const bool bact = rowok && idx < N1, aact = rowok && idx < N2;
    const size_t row = size_t(k) * N + y0 + min(r, nr - 1);
    const int yy = y0 + min(r, nr - 1);
    float* uxr = ux + row * N;
    float* uyr = uy + row * N;
    const bool zero = kind == 0 && init;
    ctx.state_ready();
    float sx[N1], sy[N1], fa[N1];
    if constexpr (STAGE) {
        if (threadIdx.x == 0) {
            const size_t r0 = (size_t(k) * N + y0) * N;
            const uint32_t bytes = rows_bytes<N>(nr);
            mbar_init(mb, 1);
            mbar_arrive_expect(mb, (zero ? 0u : 2u * bytes) + uint32_t(N * sizeof(float)));
            if (!zero) {
                bulk_load(Sx, ux + r0, bytes, mb);
                bulk_load(Sy, uy + r0, bytes, mb);
            }
            bulk_load(Sa, g.a_stag, N * sizeof(float), mb);
        }
    } else if (!LATE && aact) {
        static_for<0, N1>([&](auto I) {
            constexpr int n1 = decltype(I)::value;
            const int x = idx + N2 * n1;
            sx[n1] = zero ? 0.f : ctx.ld(uxr + x);
            sy[n1] = zero ? 0.f : ctx.ld(uyr + x);
            fa[n1] = g.a_stag[x];
        });
    }
    const float ay = g.a_stag[yy];
    F::fill_tables(twA, twB, g.tw, threadIdx.x, blockDim.x);
    ctx.input_ready();
    float2 b[N2];
    if (bact) load_c2r_b<F>(b, idx, A + row * g.hp, B + row * g.hp);
    __syncthreads();
    if (bact) F::inv_b_t(b, idx, Z0 + r * ZR, twB);
    __syncthreads();
    if constexpr (STAGE) mbar_wait(mb, 0, g.status);
    if (aact) {
        float2 a[N1];
        F::inv_a_load(a, idx, Z0 + r * ZR);
        F::inv_a(a);
        static_for<0, N1>([&](auto I) {
            constexpr int n1 = decltype(I)::value;
            const int x = idx + N2 * n1;
            const float2 gv = a[n1];
            float ax, ux0, uy0;
            if constexpr (STAGE) {
                ax = Sa[x];
                ux0 = zero ? 0.f : Sx[r * N + x];
                uy0 = zero ? 0.f : Sy[r * N + x];
            } else if constexpr (LATE) {   // fetched where used (fewer registers)
                ax = g.a_stag[x];
                ux0 = zero ? 0.f : ctx.ld(uxr + x);
                uy0 = zero ? 0.f : ctx.ld(uyr + x);
            } else {
                ax = fa[n1];
                ux0 = sx[n1];
                uy0 = sy[n1];
            }
            if (kind == 0) {
                const float uxo = init ? 0.5f * gv.x : ux0;
                const float uyo = init ? 0.5f * gv.y : uy0;
                const float uxn = ax * (ax * uxo - gv.x);
                const float uyn = ay * (ay * uyo - gv.y);
                uxr[x] = uxn;
                uyr[x] = uyn;
                if (float* ck = ctx.ck_a()) {   // checkpoint copy of u^{n+1/2} (rows of data set k)
                    const size_t o = row * N + x;
                    ck[o] = uxn;
                    ck[o + size_t(g.K) * N * N] = uyn;
                }
                a[n1] = make_float2(uxn, uyn);
            } else {
                const float tpx = ax * (ux0 + gv.x);
                const float tpy = ay * (uy0 + gv.y);
                uxr[x] = ax * tpx;
                uyr[x] = ay * tpy;
                a[n1] = make_float2(tpx, tpy);
            }
        });
        F::fwd_a_t(a, idx, Z1 + r * ZR, twA);
    }
    __syncthreads();
    finish_fwd<F>(Z1 + r * ZR, idx, bact);
    unpack_rows<F, ZR>(Z1, nr, [&](int j) { return A + (size_t(k) * N + y0 + j) * g.hp; },
                   [&](int j) { return B + (size_t(k) * N + y0 + j) * g.hp; });
}

template <int N1, int N2, int RR, bool STAGE>
__global__ void __launch_bounds__(RR * Fft2<N1, N2>::T) kf_row_u(Geo g, float2* __restrict__ A,
                                                                float2* __restrict__ B, float* __restrict__ ux,
                                                                float* __restrict__ uy, int kind, int init) {
    row_u_body<N1, N2, RR, STAGE, false>(g, LaunchedCtx{int(blockIdx.x), int(blockIdx.y)}, A, B, ux, uy, kind, init);
}

// density / pressure row pass (mode 0 regular, 1 init from p0, 2 restore), sensor gather,
// history, then A <- R2C of p (two rows per complex transform).  State, medium and PML are
// written two or more kernels earlier: fetched before the wait.
template <int N1, int N2, int RR, bool STAGE, bool LATE, class Ctx>
__device__ __forceinline__ void row_rho_body(const Geo& g, const Ctx& ctx, float2* __restrict__ A,
                                             const float2* __restrict__ B, float* __restrict__ rx,
                                             float* __restrict__ ry, const float* __restrict__ cg, int mode,
                                             const float* __restrict__ p0, float* __restrict__ y, int tstep,
                                             float* __restrict__ hist, int hist_slot) {
    using F = Fft2<N1, N2>;
    constexpr int N = F::N, T = F::T;
    constexpr int ZR = RowPad<N1, N2>::zs, PN = RowPad<N1, N2>::pn;   // padded row strides
    extern __shared__ float2 sm[];
    float2* twA = sm;       // twiddles of the A-layout step [N], read with consecutive n2 across threads
    float2* twB = sm + N;   // twiddles of the B-layout step [N], read with consecutive k1 across threads
    float2* Z0 = sm + 2 * N;
    float2* Z1 = Z0 + RR * ZR;
    float* P = reinterpret_cast<float*>(Z1 + RR * ZR);   // [RR][PN]
    float* Sx = P + RR * PN;                                // staged rho_x, rho_y, c [RR][N] each
    float* Sy = Sx + RR * N;
    float* Sc = Sy + RR * N;
    float* Sa = Sc + RR * N;                                // PML factors [N]
    uint64_t* mb = reinterpret_cast<uint64_t*>(Sa + N);
    const int k = ctx.k, y0 = ctx.bx * RR;
    const int r = threadIdx.x / T, idx = threadIdx.x % T;
    const int nr = min(RR, N - y0);
    const bool rowok = r < nr;
    const bool bact = mode == 0 && rowok && idx < N1, aact = rowok && idx < N2;
    const int yy = y0 + min(r, nr - 1);
    const size_t row = size_t(k) * N + yy;
    float* rxr = rx + row * N;
    float* ryr = ry + row * N;
    const float* cr = medium_of(g, cg, k) + size_t(yy) * N;
    const int yd = yy - g.P;
    // initial pressure at x = idx + N2 n1 (mode 1)
    auto p0_at = [&](int x) {
        const int xd = x - g.P;
        return (xd >= 0 && xd < g.n && yd >= 0 && yd < g.n) ? p0[(size_t(k) * g.n + yd) * g.n + xd] : 0.f;
    };
    float s0[N1], s1[N1], cc[N1], fa[N1];
    ctx.state_ready();
    if constexpr (STAGE) {
        if (threadIdx.x == 0) {
            const size_t r0 = (size_t(k) * N + y0) * N;
            const uint32_t bytes = rows_bytes<N>(nr);
            mbar_init(mb, 1);
            mbar_arrive_expect(mb, (mode == 1 ? 1u : 3u) * bytes + uint32_t(N * sizeof(float)));
            if (mode != 1) {
                bulk_load(Sx, rx + r0, bytes, mb);
                bulk_load(Sy, ry + r0, bytes, mb);
            }
            bulk_load(Sc, medium_of(g, cg, k) + size_t(y0) * N, bytes, mb);
            bulk_load(Sa, g.a_cell, N * sizeof(float), mb);
        }
    } else if (!LATE && aact) {
        static_for<0, N1>([&](auto I) {
            constexpr int n1 = decltype(I)::value;
            const int x = idx + N2 * n1;
            cc[n1] = cr[x];
            fa[n1] = g.a_cell[x];
            s0[n1] = mode == 1 ? p0_at(x) : ctx.ld(rxr + x);
            s1[n1] = mode == 1 ? 0.f : ctx.ld(ryr + x);
        });
    }
    const float acy = g.a_cell[yy];
    F::fill_tables(twA, twB, g.tw, threadIdx.x, blockDim.x);
    ctx.input_ready();
    float2 b[N2];
    if (bact) load_c2r_b<F>(b, idx, A + row * g.hp, B + row * g.hp);
    __syncthreads();
    if (bact) F::inv_b_t(b, idx, Z0 + r * ZR, twB);
    __syncthreads();
    if constexpr (STAGE) mbar_wait(mb, 0, g.status);
    if (aact) {
        float* Pr = P + r * PN;
        float* hr = hist ? hist + (size_t(k) * g.s_eff + in_range_or_zero(hist_slot, g.s_eff, g.status)) * N * N +
                               size_t(yy) * N
                         : nullptr;
        float2 a[N1];
        if (mode == 0) {
            F::inv_a_load(a, idx, Z0 + r * ZR);
            F::inv_a(a);
        }
        static_for<0, N1>([&](auto I) {
            constexpr int n1 = decltype(I)::value;
            const int x = idx + N2 * n1;
            float c, acx, v0, v1;
            if constexpr (STAGE) {
                c = Sc[r * N + x];
                acx = Sa[x];
                v0 = mode == 1 ? p0_at(x) : Sx[r * N + x];
                v1 = mode == 1 ? 0.f : Sy[r * N + x];
            } else if constexpr (LATE) {   // fetched where used (fewer registers)
                c = cr[x];
                acx = g.a_cell[x];
                v0 = mode == 1 ? p0_at(x) : ctx.ld(rxr + x);
                v1 = mode == 1 ? 0.f : ctx.ld(ryr + x);
            } else {
                c = cc[n1];
                acx = fa[n1];
                v0 = s0[n1];
                v1 = s1[n1];
            }
            float pv;
            if (mode == 0) {
                const float2 gv = a[n1];
                const float rxn = acx * (acx * v0 - gv.x);
                const float ryn = acy * (acy * v1 - gv.y);
                rxr[x] = rxn;
                ryr[x] = ryn;
                if (float* ck = ctx.ck_b()) {   // checkpoint copy of rho^{n+1} (rows of data set k)
                    const size_t o = row * N + x;
                    ck[o] = rxn;
                    ck[o + size_t(g.K) * N * N] = ryn;
                }
                pv = c * c * (rxn + ryn);
            } else if (mode == 1) {
                pv = v0;
                const float rv = pv / (2.f * c * c);
                rxr[x] = rv;
                ryr[x] = rv;
            } else {
                pv = c * c * (v0 + v1);
            }
            Pr[x] = pv;
            if (hr) hr[x] = pv;
        });
    }
    __syncthreads();
    if (y) {
        const int e0 = g.srow[y0], e1 = g.srow[y0 + nr];
        for (int e = e0 + threadIdx.x; e < e1; e += blockDim.x) {
            const int2 se = g.sent[e];
            const float4 sw = g.sentw[e];
            const int rr = int(sw.w) - y0;
            if (!(in_range(rr, nr, g.status) && in_range(se.y + 1, N, g.status) && in_range(se.x, g.m, g.status) &&
                  in_range(tstep, g.nt, g.status)))
                continue;
            const float v = sw.z * (sw.x * P[rr * PN + se.y] + sw.y * P[rr * PN + se.y + 1]);
            // at most two adds (rows iy, iy+1) onto a zeroed sample: order-independent
            atomicAdd(&y[(size_t(k) * g.nt + tstep) * g.m + se.x], v);
        }
    }
    const int np = nr / 2;
    const bool pairok = r < np;
    if (pairok && idx < N2) {
        float2 a[N1];
        static_for<0, N1>([&](auto I) {
            constexpr int n1 = decltype(I)::value;
            const int x = N2 * n1 + idx;
            a[n1] = make_float2(P[(2 * r) * PN + x], P[(2 * r + 1) * PN + x]);
        });
        F::fwd_a_t(a, idx, Z1 + r * ZR, twA);
    }
    __syncthreads();
    finish_fwd<F>(Z1 + r * ZR, idx, pairok && idx < N1);
    unpack_rows<F, ZR>(Z1, np, [&](int j) { return A + (size_t(k) * N + y0 + 2 * j) * g.hp; },
                   [&](int j) { return A + (size_t(k) * N + y0 + 2 * j + 1) * g.hp; });
}

template <int N1, int N2, int RR, bool STAGE>
__global__ void __launch_bounds__(RR * Fft2<N1, N2>::T) kf_row_rho(Geo g, float2* __restrict__ A,
                                                                  const float2* __restrict__ B,
                                                                  float* __restrict__ rx, float* __restrict__ ry,
                                                                  const float* __restrict__ cg, int mode,
                                                                  const float* __restrict__ p0,
                                                                  float* __restrict__ y, int tstep,
                                                                  float* __restrict__ hist, int hist_slot) {
    row_rho_body<N1, N2, RR, STAGE, false>(g, LaunchedCtx{int(blockIdx.x), int(blockIdx.y)}, A, B, rx, ry, cg, mode, p0,
                                    y, tstep, hist, hist_slot);
}

// adjoint density row pass: pb = C2R(Q) + S^T r^n; rb += c^2 pb; cbar += 2 p pb / c;
// t = a rb; rb <- a t; (A2, B2) <- R2C(t_x, t_y).  Adjoint state, dJ/dc accumulator,
// medium, PML, pressure history and sensor source are fetched before the wait; the spectrum,
// written by the preceding kernel, after it.
template <int N1, int N2, int RR, bool STAGE>
__global__ void __launch_bounds__(RR * Fft2<N1, N2>::T) kf_row_adj_rho(Geo g, float2* __restrict__ A2,
                                                                      float2* __restrict__ B2,
                                                                      float* __restrict__ rbx,
                                                                      float* __restrict__ rby,
                                                                      float* __restrict__ cbar,
                                                                      const float* __restrict__ cg, int first,
                                                                      const float* __restrict__ resid, int tstep,
                                                                      const float* __restrict__ hist,
                                                                      int hist_slot) {
    using F = Fft2<N1, N2>;
    constexpr int N = F::N, T = F::T;
    constexpr int ZR = RowPad<N1, N2>::zs, PN = RowPad<N1, N2>::pn;   // padded row strides
    extern __shared__ float2 sm[];
    float2* twA = sm;       // twiddles of the A-layout step [N], read with consecutive n2 across threads
    float2* twB = sm + N;   // twiddles of the B-layout step [N], read with consecutive k1 across threads
    float2* Z0 = sm + 2 * N;
    float2* Z1 = Z0 + RR * ZR;
    float* PB = reinterpret_cast<float*>(Z1 + RR * ZR);   // [RR][PN]
    float* Sx = PB + RR * PN;                                // staged rb_x, rb_y, c, p history [RR][N] each
    float* Sy = Sx + RR * N;
    float* Sc = Sy + RR * N;
    float* Sh = Sc + RR * N;
    float* Sa = Sh + RR * N;                                 // PML factors [N]
    float* Sb = Sa + N;                                      // dJ/dc rows of the domain [RR][n]
    uint64_t* mb = reinterpret_cast<uint64_t*>(Sb + RR * g.n);
    const int k = blockIdx.y, y0 = blockIdx.x * RR;
    const int r = threadIdx.x / T, idx = threadIdx.x % T;
    const int nr = min(RR, N - y0);
    const bool rowok = r < nr;
    const int np = nr / 2;
    const bool pairok = r < np;
    const bool bact = !first && pairok && idx < N1, aact = rowok && idx < N2;
    const int yy = y0 + min(r, nr - 1);
    const size_t row = size_t(k) * N + yy;
    const int yd = yy - g.P;
    const bool yin = yd >= 0 && yd < g.n;
    float* bx = rbx + row * N;
    float* by = rby + row * N;
    float* cbr = cbar + (size_t(k) * g.n + (yin ? yd : 0)) * g.n;
    const float* cr = medium_of(g, cg, k) + size_t(yy) * N;
    // domain rows of the tile in dJ/dc (staged when a row is a multiple of 16 bytes)
    const int d0 = max(y0 - g.P, 0), d1 = min(y0 + nr - g.P, g.n);
    const bool cb_staged = STAGE && (g.n % 4) == 0;
    float s0[N1], s1[N1], cc[N1], hv[N1], fa[N1], cb[N1];
    if constexpr (STAGE) {
        if (threadIdx.x == 0) {
            const size_t r0 = (size_t(k) * N + y0) * N;
            const uint32_t bytes = rows_bytes<N>(nr);
            const uint32_t cbytes = (cb_staged && d1 > d0) ? uint32_t(d1 - d0) * g.n * sizeof(float) : 0u;
            mbar_init(mb, 2);   // this arrival and the history's
            mbar_arrive_expect(mb, 3u * bytes + uint32_t(N * sizeof(float)) + cbytes);
            bulk_load(Sx, rbx + r0, bytes, mb);
            bulk_load(Sy, rby + r0, bytes, mb);
            bulk_load(Sc, medium_of(g, cg, k) + size_t(y0) * N, bytes, mb);
            bulk_load(Sa, g.a_cell, N * sizeof(float), mb);
            if (cbytes) bulk_load(Sb, cbar + (size_t(k) * g.n + d0) * g.n, cbytes, mb);
        }
    } else if (aact) {
        static_for<0, N1>([&](auto I) {
            constexpr int n1 = decltype(I)::value;
            const int x = idx + N2 * n1;
            const int xd = x - g.P;
            s0[n1] = bx[x];
            s1[n1] = by[x];
            cc[n1] = cr[x];
            fa[n1] = g.a_cell[x];
            cb[n1] = (yin && xd >= 0 && xd < g.n) ? cbr[xd] : 0.f;
        });
    }
    const float acy = g.a_cell[yy];
    F::fill_tables(twA, twB, g.tw, threadIdx.x, blockDim.x);
    if (first)
        for (int i = threadIdx.x; i < RR * PN; i += blockDim.x) PB[i] = 0.f;
    // The source S^T r^n of the tile's rows, fetched before the wait (the residual is written
    // before the reverse sweep starts): per sensor entry its column and its two weighted values,
    // so that the in-order accumulation after the inverse transform reads only shared memory.
    constexpr int kMaxEnt = 16 * RR;
    __shared__ int s_ecol[kMaxEnt];
    __shared__ float s_ewa[kMaxEnt], s_ewb[kMaxEnt];
    const int e0 = g.srow[y0], e1 = g.srow[y0 + nr];
    const bool ent_pre = e1 - e0 <= kMaxEnt;
    const float* rv = resid + (size_t(k) * g.nt + in_range_or_zero(tstep, g.nt, g.status)) * g.m;
    if (ent_pre)
        for (int e = e0 + int(threadIdx.x); e < e1; e += blockDim.x) {
            const int2 se = g.sent[e];
            const float4 sw = g.sentw[e];
            const bool ok = in_range(se.x, g.m, g.status) && in_range(se.y + 1, N, g.status);
            const float v = ok ? rv[se.x] * sw.z : 0.f;
            s_ecol[e - e0] = ok ? se.y : 0;
            s_ewa[e - e0] = sw.x * v;
            s_ewb[e - e0] = sw.y * v;
        }
    // The pressure history is written by the segment recompute on the other stream, which this
    // segment's first kernel waits for through an event (a full dependency), or by the forward
    // sweep: never by the kernel just before, so it is fetched before the wait as well.
    const int hslot = in_range_or_zero(hist_slot, g.s_eff, g.status);
    const float* hr = hist + (size_t(k) * g.s_eff + hslot) * N * N + size_t(yy) * N;
    if constexpr (STAGE) {
        if (threadIdx.x == 0) {
            const uint32_t bytes = rows_bytes<N>(nr);
            mbar_arrive_expect(mb, bytes);
            bulk_load(Sh, hist + (size_t(k) * g.s_eff + hslot) * N * N + size_t(y0) * N, bytes, mb);
        }
    } else if (aact) {
        static_for<0, N1>([&](auto I) { hv[decltype(I)::value] = hr[idx + N2 * decltype(I)::value]; });
    }
    pdl_wait_then_release();
    float2 b[N2];
    if (bact) {
        const float2* q0 = A2 + (size_t(k) * N + y0 + 2 * r) * g.hp;
        load_c2r_b<F>(b, idx, q0, q0 + g.hp);
    }
    __syncthreads();
    if (bact) F::inv_b_t(b, idx, Z0 + r * ZR, twB);
    __syncthreads();
    if (!first && pairok && idx < N2) {
        float2 a[N1];
        F::inv_a_load(a, idx, Z0 + r * ZR);
        F::inv_a(a);
        static_for<0, N1>([&](auto I) {
            constexpr int n1 = decltype(I)::value;
            const int x = idx + N2 * n1;
            PB[(2 * r) * PN + x] = a[n1].x;
            PB[(2 * r + 1) * PN + x] = a[n1].y;
        });
    }
    __syncthreads();
    if (threadIdx.x < nr) {   // S^T r^n, one thread per row: fixed order
        const int rr = threadIdx.x, yr = y0 + rr;
        const int ea = g.srow[yr], eb = g.srow[yr + 1];
        if (ent_pre) {
            for (int e = ea; e < eb; ++e) {
                const int col = s_ecol[e - e0];
                PB[rr * PN + col] += s_ewa[e - e0];
                PB[rr * PN + col + 1] += s_ewb[e - e0];
            }
        } else {
            for (int e = ea; e < eb; ++e) {
                const int2 se = g.sent[e];
                const float4 sw = g.sentw[e];
                if (!(in_range(se.x, g.m, g.status) && in_range(se.y + 1, N, g.status))) continue;
                const float v = rv[se.x] * sw.z;
                PB[rr * PN + se.y] += sw.x * v;
                PB[rr * PN + se.y + 1] += sw.y * v;
            }
        }
    }
    __syncthreads();
    if constexpr (STAGE) mbar_wait(mb, 0, g.status);
    if (aact) {
        float2 a[N1];
        static_for<0, N1>([&](auto I) {
            constexpr int n1 = decltype(I)::value;
            const int x = idx + N2 * n1;
            const int xd = x - g.P;
            const bool xin = yin && xd >= 0 && xd < g.n;
            float v0, v1, c, acx, cbo, h;
            if constexpr (STAGE) {
                v0 = Sx[r * N + x];
                v1 = Sy[r * N + x];
                c = Sc[r * N + x];
                acx = Sa[x];
                h = Sh[r * N + x];
                cbo = xin ? (cb_staged ? Sb[(yd - d0) * g.n + xd] : cbr[xd]) : 0.f;
            } else {
                v0 = s0[n1];
                v1 = s1[n1];
                c = cc[n1];
                acx = fa[n1];
                cbo = cb[n1];
                h = hv[n1];
            }
            const float p_b = PB[r * PN + x];
            const float c2 = c * c;
            const float vbx = v0 + c2 * p_b;
            const float vby = v1 + c2 * p_b;
            if (xin) cbr[xd] = cbo + 2.f * h * p_b / c;
            const float tx = acx * vbx, ty = acy * vby;
            bx[x] = acx * tx;
            by[x] = acy * ty;
            a[n1] = make_float2(tx, ty);
        });
        F::fwd_a_t(a, idx, Z1 + r * ZR, twA);
    }
    __syncthreads();
    finish_fwd<F>(Z1 + r * ZR, idx, rowok && idx < N1);
    unpack_rows<F, ZR>(Z1, nr, [&](int j) { return A2 + (size_t(k) * N + y0 + j) * g.hp; },
                   [&](int j) { return B2 + (size_t(k) * N + y0 + j) * g.hp; });
}

// ---------------------------------------------------------------------------
// launch with programmatic stream serialisation (the kernel calls pdl_wait_then_release)
// (pdl = false: an ordinary launch, used after copies and memsets)
template <typename... KArgs, typename... Args>
inline void launch_pdl(void (*kern)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t st, bool pdl,
                       Args... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = pdl ? 1 : 0;
    cudaLaunchKernelEx(&cfg, kern, args...);
}

template <int N1, int N2, int RR, int CC, bool STAGE>
struct FixedImpl {
    using F = Fft2<N1, N2>;
    static constexpr int n1 = N1, n2 = N2, rr = RR, cc = CC;
    using RS = RowSmem<F, RR>;
    static constexpr size_t smem_col = ColSmem<N1, N2, CC>::bytes;
    static_assert(2 * F::ZS >= F::ZS + F::N1 * F::N2, "product hand-off fits the inverse buffer");
    static_assert(!STAGE || (F::N % 4 == 0 && RR % 2 == 0), "staged row blocks are 16-byte multiples");
    // staged: velocity 2 arrays, density 3, adjoint density 4 and the dJ/dc rows (n < Ng)
    static constexpr size_t smem_u = STAGE ? RS::staged(2, 0, 0) : RS::base;
    static constexpr size_t smem_rho = STAGE ? RS::staged(3, 0, 0) : RS::base;
    static constexpr size_t smem_adj = STAGE ? RS::staged(4, 1, F::N) : RS::base;

    static int configure() {
        cudaError_t e = cudaFuncSetAttribute((const void*)kf_col<N1, N2, CC>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem_col));
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute((const void*)kf_row_u<N1, N2, RR, STAGE>,
                                     cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem_u));
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute((const void*)kf_row_rho<N1, N2, RR, STAGE>,
                                     cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem_rho));
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute((const void*)kf_row_adj_rho<N1, N2, RR, STAGE>,
                                     cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem_adj));
        return e == cudaSuccess ? PAT_OK : cuda_fail(e, "cudaFuncSetAttribute(fixed-size kernels)");
    }
    static void col(const Geo& g, cudaStream_t st, float2* A, float2* B, int mode, int op, float scale) {
        dim3 grid((g.hc + CC - 1) / CC, g.K);
        launch_pdl(kf_col<N1, N2, CC>, grid, dim3(2 * CC * F::T), smem_col, st, true, g, A, B, mode, op, scale);
    }
    static void row_u(const Geo& g, cudaStream_t st, float2* A, float2* B, float* ux, float* uy, int kind,
                      int init) {
        dim3 grid((F::N + RR - 1) / RR, g.K);
        launch_pdl(kf_row_u<N1, N2, RR, STAGE>, grid, dim3(RR * F::T), smem_u, st, true, g, A, B, ux, uy, kind,
                   init);
    }
    static void row_rho(const Geo& g, cudaStream_t st, float2* A, const float2* B, float* rx, float* ry,
                        const float* cg, int mode, const float* p0, float* y, int tstep, float* hist, int slot) {
        dim3 grid((F::N + RR - 1) / RR, g.K);
        launch_pdl(kf_row_rho<N1, N2, RR, STAGE>, grid, dim3(RR * F::T), smem_rho, st, mode == 0, g, A, B, rx, ry,
                   cg, mode, p0, y, tstep, hist, slot);
    }
    static void row_adj_rho(const Geo& g, cudaStream_t st, float2* A2, float2* B2, float* rbx, float* rby,
                            float* cbar, const float* cg, int first, const float* resid, int tstep,
                            const float* hist, int slot) {
        dim3 grid((F::N + RR - 1) / RR, g.K);
        launch_pdl(kf_row_adj_rho<N1, N2, RR, STAGE>, grid, dim3(RR * F::T), smem_adj, st, true, g, A2, B2, rbx,
                   rby, cbar, cg, first, resid, tstep, hist, slot);
    }
    static FixedOps ops() {
        return FixedOps{F::N, RR, CC, &configure, &col, &row_u, &row_rho, &row_adj_rho, nullptr, nullptr, nullptr};
    }
};

// Column passes on the three-level transform (only the column pass of the launch table;
// combined with row passes of other impls through MixedImpl).
template <int NA, int NM, int NB, int CC>
struct Col3Impl {
    using F = Fft3<NA, NM, NB>;
    static constexpr int cc = CC;
    static constexpr size_t smem_col = (F::N + F::N2 + 2 * F::N * CC + 4 * F::ZS * CC) * sizeof(float2);
    static_assert(F::ZS >= F::N, "product hand-off fits one field's buffer");
    static int configure() {
        cudaError_t e = cudaFuncSetAttribute((const void*)kf_col3<NA, NM, NB, CC>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem_col));
        return e == cudaSuccess ? PAT_OK : cuda_fail(e, "cudaFuncSetAttribute(kf_col3)");
    }
    static void col(const Geo& g, cudaStream_t st, float2* A, float2* B, int mode, int op, float scale) {
        dim3 grid((g.hc + CC - 1) / CC, g.K);
        launch_pdl(kf_col3<NA, NM, NB, CC>, grid, dim3(2 * CC * F::T), smem_col, st, true, g, A, B, mode, op,
                   scale);
    }
};

// Column passes with the multipliers formed where they are used (col_body LEAN; only the column
// pass of the launch table, combined with row passes of other impls through MixedImpl).
template <int N1, int N2, int CC>
struct ColLeanImpl {
    using F = Fft2<N1, N2>;
    static constexpr int cc = CC;
    static constexpr size_t smem_col = ColSmem<N1, N2, CC, true>::bytes;
    static int configure() {
        cudaError_t e = cudaFuncSetAttribute((const void*)kf_col_lean<N1, N2, CC>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem_col));
        return e == cudaSuccess ? PAT_OK : cuda_fail(e, "cudaFuncSetAttribute(kf_col_lean)");
    }
    static void col(const Geo& g, cudaStream_t st, float2* A, float2* B, int mode, int op, float scale) {
        dim3 grid((g.hc + CC - 1) / CC, g.K);
        launch_pdl(kf_col_lean<N1, N2, CC>, grid, dim3(2 * CC * F::T), smem_col, st, true, g, A, B, mode, op,
                   scale);
    }
};

// A variant whose pass kinds come from different tile shapes / factorisations of the same
// Ng (the half spectra in global memory have one layout): column passes from C (from CS when
// the pass runs alone on the GPU), velocity row passes from U, density row passes from R,
// adjoint density row passes from J; the segment recompute's velocity and density row passes
// from RU and RR when given (void: U and R).
template <class C, class U, class R, class J, class CS = C, class RU = void, class RR = void>
struct MixedImpl {
    static_assert(C::F::N == U::F::N && C::F::N == R::F::N && C::F::N == J::F::N && C::F::N == CS::F::N,
                  "one grid side");
    static int configure() {
        int rc = C::configure();
        if (rc == PAT_OK) rc = U::configure();
        if (rc == PAT_OK) rc = R::configure();
        if (rc == PAT_OK) rc = J::configure();
        if (rc == PAT_OK) rc = CS::configure();
        if constexpr (!std::is_void_v<RU>) {
            if (rc == PAT_OK) rc = RU::configure();
        }
        if constexpr (!std::is_void_v<RR>) {
            if (rc == PAT_OK) rc = RR::configure();
        }
        return rc;
    }
    static FixedOps ops() {
        FixedOps o{C::F::N, 0, 0, &configure, &C::col, &U::row_u, &R::row_rho, &J::row_adj_rho, &CS::col,
                   nullptr, nullptr};
        if constexpr (!std::is_void_v<RU>) o.row_u_rc = &RU::row_u;
        if constexpr (!std::is_void_v<RR>) o.row_rho_rc = &RR::row_rho;
        return o;
    }
};

// ---------------------------------------------------------------------------
// Persistent forward sweep: one launch runs the initial pass and all Nt-1 steps of every
// data set of the plan (all instances of a batch).  The passes of the sweep are cut into
// work items (pass q, data set k, tile b), numbered pass by pass and, within a pass, data
// set by data set; CTAs take item numbers from a counter in the workspace (a ticket queue)
// and run the same pass bodies as the launched passes.  An item waits only for the items
// of its own data set in the passes before it (a per-data-set counter of completed items),
// so data sets advance independently and a pass of one data set overlaps the tail of
// another's.  Every item a CTA waits for has a smaller number and was taken earlier by a
// running CTA, and the smallest unfinished item never waits, so the sweep progresses
// whatever the number of resident CTAs.  Each wait is bounded: after kQueueWaitNs it sets
// PAT_STATUS_QUEUE in the workspace status word and an abort flag that ends every later
// wait at once (the results of that sweep are then invalid; no hang).
struct SweepArgs {
    float2* A;
    float2* B;
    float *ux, *uy, *rx, *ry;   // state [K][ng][ng] each (contiguous, ux first)
    const float* cg;            // c on the grid [ninst][ng][ng]
    const float* p0;            // [K][n][n]
    float* y;                   // traces [K][nt][m], zeroed
    float* hist;                // pressure history of the last segment (levels >= last0), or null
    int last0;
    float* ckpt;                // checkpoints [slot][4][K][ng][ng] at levels j s (slot j-1), or null
    int s;
    float sg, sd;               // scales of the G and D multipliers
    int nsteps;                 // Nt - 1
    int* queue;                 // [0] ticket counter, [1] abort flag, [2 + k] items done of data set k
    unsigned long long wait_ns; // limit of one dependency wait
};

constexpr unsigned long long kQueueWaitNs = 1000000000ull;
constexpr int kStatusQueue = 4;   // PAT_STATUS_QUEUE

struct QueueCtx {
    int bx, k;
    int need_state, need_input;   // items of data set k that must be done at each dependency point
    int* queue;
    int* status;
    float* cka;                   // checkpoint targets of the velocity / density rows, or null
    float* ckb;
    unsigned long long wait_ns;
    // state rows written by other CTAs of the same launch: L2 loads (the SM's L1 may hold old lines)
    __device__ __forceinline__ float ld(const float* p) const { return __ldcg(p); }
    __device__ __forceinline__ void wait(int need) const {
        if (threadIdx.x == 0) {
            const volatile int* done = queue + 2 + k;
            const volatile int* abort_flag = queue + 1;
            if (*done < need && !*abort_flag) {
                const uint64_t t0 = global_ns();
                while (*done < need && !*abort_flag) {
                    if (global_ns() - t0 > wait_ns) {
                        if (status) atomicOr(status, kStatusQueue);
                        atomicExch(queue + 1, 1);
                        break;
                    }
                    __nanosleep(64);
                }
            }
            __threadfence();
        }
        __syncthreads();
    }
    __device__ __forceinline__ void state_ready() const { wait(need_state); }
    __device__ __forceinline__ void input_ready() const { wait(need_input); }
    __device__ __forceinline__ float* ck_a() const { return cka; }
    __device__ __forceinline__ float* ck_b() const { return ckb; }
};

// C: column passes, U: velocity row passes, R: density row passes (one thread count)
template <class C, class U, class R>
struct PersistentImpl {
    static constexpr int N = C::F::N;
    static constexpr int NT = 2 * C::cc * C::F::T;
    static_assert(U::F::N == N && R::F::N == N, "one grid side");
    static_assert(U::rr * U::F::T == NT && R::rr * R::F::T == NT && U::rr == R::rr, "one thread count");
    static constexpr int RR = U::rr, CC = C::cc;
    static constexpr int MINB = 2;   // CTAs per SM the register budget is cut for
    static constexpr size_t smem = C::smem_col > U::smem_u ? (C::smem_col > R::smem_rho ? C::smem_col : R::smem_rho)
                                                           : (U::smem_u > R::smem_rho ? U::smem_u : R::smem_rho);
    static int blocks_per_sm;

    // The row bodies fetch the state where they use it (LATE): other CTAs of the sweep hide
    // that latency.  The bodies are outlined (each its own register allocation): inlined
    // into one item loop, values shared across them stay live at once and spill.
    static __device__ __noinline__ void init_pass(const Geo& g, const QueueCtx& ctx, const SweepArgs& a) {
        row_rho_body<R::n1, R::n2, RR, false, true>(g, ctx, a.A, a.B, a.rx, a.ry, a.cg, 1, a.p0, a.y, 0,
                                              (a.hist && a.last0 == 0) ? a.hist : nullptr, 0);
    }
    static __device__ __noinline__ void col_pass(const Geo& g, const QueueCtx& ctx, const SweepArgs& a, int op) {
        col_body<C::n1, C::n2, CC>(g, ctx, a.A, a.B, op, op, op ? a.sd : a.sg);
    }
    static __device__ __noinline__ void u_pass(const Geo& g, const QueueCtx& ctx, const SweepArgs& a, int init) {
        row_u_body<U::n1, U::n2, RR, false, true>(g, ctx, a.A, a.B, a.ux, a.uy, 0, init);
    }
    static __device__ __noinline__ void rho_pass(const Geo& g, const QueueCtx& ctx, const SweepArgs& a, int lv) {
        const bool h = a.hist && lv >= a.last0;
        row_rho_body<R::n1, R::n2, RR, false, true>(g, ctx, a.A, a.B, a.rx, a.ry, a.cg, 0, nullptr, a.y, lv,
                                              h ? a.hist : nullptr, lv - a.last0);
    }

    static __device__ __forceinline__ void run(const Geo& g, const SweepArgs& a) {
        const int K = g.K;
        const int nbc = (g.hc + CC - 1) / CC, nbr = (N + RR - 1) / RR;
        const int per_k_step = 2 * nbc + 2 * nbr;
        const int per_step = K * per_k_step;
        const int total = K * nbr + per_step * a.nsteps;
        const size_t f = size_t(K) * N * N;
        __shared__ int s_item;
        for (;;) {
            __syncthreads();   // the previous item is finished with shared memory and s_item
            if (threadIdx.x == 0) s_item = atomicAdd(a.queue, 1);
            __syncthreads();
            const int item = s_item;
            if (item >= total) return;
            QueueCtx ctx{0, 0, 0, 0, a.queue, g.status, nullptr, nullptr, a.wait_ns};
            if (item < K * nbr) {   // initial condition from p0
                ctx.k = item / nbr;
                ctx.bx = item - ctx.k * nbr;
                init_pass(g, ctx, a);
            } else {
                const int i2 = item - K * nbr;
                const int n = i2 / per_step;
                int r = i2 - n * per_step;
                int p, pre, prev;
                if (r < K * nbc) {
                    p = 0; pre = 0; prev = nbr;
                    ctx.k = r / nbc; ctx.bx = r - ctx.k * nbc;
                } else if ((r -= K * nbc) < K * nbr) {
                    p = 1; pre = nbc; prev = nbc;
                    ctx.k = r / nbr; ctx.bx = r - ctx.k * nbr;
                } else if ((r -= K * nbr) < K * nbc) {
                    p = 2; pre = nbc + nbr; prev = nbr;
                    ctx.k = r / nbc; ctx.bx = r - ctx.k * nbc;
                } else {
                    r -= K * nbc;
                    p = 3; pre = 2 * nbc + nbr; prev = nbc;
                    ctx.k = r / nbr; ctx.bx = r - ctx.k * nbr;
                }
                ctx.need_input = nbr + n * per_k_step + pre;
                ctx.need_state = ctx.need_input - prev;
                const int lv = n + 1;   // level written by this step
                float* ck = (a.ckpt && lv % a.s == 0) ? a.ckpt + size_t(lv / a.s - 1) * 4 * f : nullptr;
                if (p == 0 || p == 2) {
                    col_pass(g, ctx, a, p == 2 ? 1 : 0);
                } else if (p == 1) {
                    ctx.cka = ck;
                    u_pass(g, ctx, a, n == 0 ? 1 : 0);
                } else {
                    ctx.ckb = ck ? ck + 2 * f : nullptr;
                    rho_pass(g, ctx, a, lv);
                }
            }
            __syncthreads();
            if (threadIdx.x == 0) {
                __threadfence();
                atomicAdd(a.queue + 2 + ctx.k, 1);
            }
        }
    }
};

template <class C, class U, class R>
int PersistentImpl<C, U, R>::blocks_per_sm = 0;

template <class P>
__global__ void __launch_bounds__(P::NT, P::MINB) kp_forward(Geo g, SweepArgs a) {
    P::run(g, a);
}

// launch table of the persistent sweep of one grid side
struct SweepOps {
    int ng;
    int (*configure)();
    int (*launch)(const Geo&, cudaStream_t, const SweepArgs&);
    int (*items)(const Geo&, int nsteps);
};

template <class P>
struct SweepImpl {
    static int configure() {
        cudaError_t e = cudaFuncSetAttribute((const void*)kp_forward<P>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             int(P::smem));
        if (e == cudaSuccess && P::blocks_per_sm == 0)
            e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&P::blocks_per_sm, kp_forward<P>, P::NT, P::smem);
        if (e == cudaSuccess && P::blocks_per_sm < 1) return cuda_fail(cudaErrorInvalidConfiguration, "kp_forward");
        return e == cudaSuccess ? PAT_OK : cuda_fail(e, "cudaFuncSetAttribute(kp_forward)");
    }
    static int items(const Geo& g, int nsteps) {
        const int nbc = (g.hc + P::CC - 1) / P::CC, nbr = (P::N + P::RR - 1) / P::RR;
        return g.K * nbr + g.K * (2 * nbc + 2 * nbr) * nsteps;
    }
    static int launch(const Geo& g, cudaStream_t st, const SweepArgs& a) {
        int dev = 0, sms = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        const int grid = std::max(1, std::min(items(g, a.nsteps), P::blocks_per_sm * std::max(sms, 1)));
        kp_forward<P><<<grid, P::NT, P::smem, st>>>(g, a);
        return PAT_OK;
    }
    static SweepOps ops() { return SweepOps{P::N, &configure, &launch, &items}; }
};

const SweepOps* sweep_ops_for(int ng);   // nullptr if the side has no persistent sweep

}  // namespace pat

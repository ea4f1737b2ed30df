// Two-level register FFT for a compile-time length N = N1 * N2 (both small,
// 5-smooth).  A length-N transform is split as in the Cooley-Tukey
// factorisation
//   X[k1 + N1 k2] = sum_{n2} W_{N2}^{n2 k2} W_N^{n2 k1} sum_{n1} x[N2 n1 + n2] W_{N1}^{n1 k1}
// so that one thread ("A layout", index n2) holds x[N2 n1 + n2] for all n1
// and does a register DFT of length N1, and after one shared-memory
// transpose another thread ("B layout", index k1) holds the values for all n2
// and does a register DFT of length N2, ending with X[k1 + N1 k2].  The
// inverse runs the same two steps backwards (B layout -> A layout), so a
// forward transform, a pointwise product in wavenumber space and an inverse
// transform need only two shared-memory transposes.
//
// Register DFTs of composite lengths are built recursively from radix 2/3/4/5
// with twiddles evaluated at compile time (constexpr Taylor series).
#pragma once

#include <cuda_runtime.h>

#include <type_traits>

#include "fft.cuh"

namespace pat {

// ---- compile-time trigonometry (Taylor series after reduction to [-pi, pi]) ----
__host__ __device__ constexpr double ce_reduce(double a) {
    constexpr double PI = 3.14159265358979323846264338327950288;
    while (a > PI) a -= 2.0 * PI;
    while (a < -PI) a += 2.0 * PI;
    return a;
}
__host__ __device__ constexpr double ce_sin(double a) {
    a = ce_reduce(a);
    double term = a, sum = a;
    for (int k = 1; k < 30; ++k) {
        term *= -a * a / double((2 * k) * (2 * k + 1));
        sum += term;
    }
    return sum;
}
__host__ __device__ constexpr double ce_cos(double a) {
    a = ce_reduce(a);
    double term = 1.0, sum = 1.0;
    for (int k = 1; k < 30; ++k) {
        term *= -a * a / double((2 * k - 1) * (2 * k));
        sum += term;
    }
    return sum;
}

template <int B, int E, class F>
__host__ __device__ __forceinline__ void static_for(F&& f) {
    if constexpr (B < E) {
        f(std::integral_constant<int, B>{});
        static_for<B + 1, E>(f);
    }
}

// z * W_N^E, W_N = exp(-2 pi i / N) (forward) or exp(+2 pi i / N) (inverse); E compile-time
template <int N, int E, bool INV>
__host__ __device__ __forceinline__ float2 twc(float2 z) {
    constexpr int e = E % N;
    if constexpr (e == 0) {
        return z;
    } else if constexpr (2 * e == N) {
        return make_float2(-z.x, -z.y);
    } else if constexpr (4 * e == N) {
        return rot<INV>(z);
    } else if constexpr (4 * e == 3 * N) {
        return rot<!INV>(z);
    } else {
        constexpr double PI = 3.14159265358979323846264338327950288;
        constexpr double a = (INV ? 2.0 : -2.0) * PI * double(e) / double(N);
        constexpr float c = float(ce_cos(a));
        constexpr float s = float(ce_sin(a));
        return make_float2(z.x * c - z.y * s, z.x * s + z.y * c);
    }
}

template <int N, bool INV>
__host__ __device__ __forceinline__ void dft(float2 (&v)[N]);

// N = A * B: DFT_A over a of v[B a + b] for each b, twiddle W_N^{b ka}, DFT_B over b
template <int A, int B, bool INV>
__host__ __device__ __forceinline__ void dft_ab(float2 (&v)[A * B]) {
    constexpr int N = A * B;
    float2 t[N];
    static_for<0, B>([&](auto bI) {
        constexpr int b = decltype(bI)::value;
        float2 u[A];
        static_for<0, A>([&](auto aI) { u[decltype(aI)::value] = v[B * decltype(aI)::value + b]; });
        dft<A, INV>(u);
        static_for<0, A>([&](auto kI) {
            constexpr int ka = decltype(kI)::value;
            t[ka * B + b] = twc<N, b * ka, INV>(u[ka]);
        });
    });
    static_for<0, A>([&](auto kI) {
        constexpr int ka = decltype(kI)::value;
        float2 u[B];
        static_for<0, B>([&](auto bI) { u[decltype(bI)::value] = t[ka * B + decltype(bI)::value]; });
        dft<B, INV>(u);
        static_for<0, B>([&](auto kbI) { v[ka + A * decltype(kbI)::value] = u[decltype(kbI)::value]; });
    });
}

template <int N, bool INV>
__host__ __device__ __forceinline__ void dft(float2 (&v)[N]) {
    if constexpr (N == 1) {
    } else if constexpr (N == 2 || N == 3 || N == 4 || N == 5) {
        dft_small<N, INV>(v);
    } else if constexpr (N % 4 == 0) {
        dft_ab<4, N / 4, INV>(v);
    } else if constexpr (N % 2 == 0) {
        dft_ab<2, N / 2, INV>(v);
    } else if constexpr (N % 3 == 0) {
        dft_ab<3, N / 3, INV>(v);
    } else {
        static_assert(N % 5 == 0, "length must be 5-smooth");
        dft_ab<5, N / 5, INV>(v);
    }
}

// Shapes of the two-level transform of length N = N1 * N2.
template <int N1_, int N2_>
struct Fft2 {
    static constexpr int N1 = N1_;
    static constexpr int N2 = N2_;
    static constexpr int N = N1 * N2;
    static constexpr int T = N1 > N2 ? N1 : N2;   // threads per sequence
    static constexpr int P2 = (N2 % 2) ? N2 : N2 + 1;   // padded row of the transpose buffer
    static constexpr int ZS = N1 * P2;            // transpose buffer elements per sequence
    // layouts in the terms shared with Fft3: A layout = AV values (x[AT n1 + idx]) in each of
    // AT threads, B layout = BV values (X[idx + BT k2]) in each of BT threads
    static constexpr int kLevels = 2;
    static constexpr int AV = N1, AT = N2, BV = N2, BT = N1;

    // Z element (k1, n2) lives at Z[(k1 P2 + n2) S] (S interleaves several transforms).
    // forward, A layout: a[n1] = x[N2 n1 + n2] -> a[k1] twiddled, stored to Z(k1, n2)
    template <int S = 1>
    __host__ __device__ static __forceinline__ void fwd_a(float2 (&a)[N1], int n2, float2* Z, const float2* tw) {
        dft<N1, false>(a);
        static_for<0, N1>([&](auto kI) {
            constexpr int k1 = decltype(kI)::value;
            float2 v = a[k1];
            if constexpr (k1 > 0) v = cmul(v, tw[n2 * k1]);
            Z[(k1 * P2 + n2) * S] = v;
        });
    }
    // forward, B layout: b[n2] = Z[k1 P2 + n2] -> b[k2] = X[k1 + N1 k2]
    template <int S = 1>
    __host__ __device__ static __forceinline__ void fwd_b_load(float2 (&b)[N2], int k1, const float2* Z) {
        static_for<0, N2>([&](auto nI) { b[decltype(nI)::value] = Z[(k1 * P2 + decltype(nI)::value) * S]; });
    }
    __host__ __device__ static __forceinline__ void fwd_b(float2 (&b)[N2]) { dft<N2, false>(b); }
    // inverse, B layout: b[k2] = X[k1 + N1 k2] -> inverse DFT_N2, twiddle, Z[k1 P2 + n2]
    template <int S = 1>
    __host__ __device__ static __forceinline__ void inv_b(float2 (&b)[N2], int k1, float2* Z, const float2* tw) {
        dft<N2, true>(b);
        static_for<0, N2>([&](auto nI) {
            constexpr int n2 = decltype(nI)::value;
            float2 v = b[n2];
            if constexpr (n2 > 0) v = cmulc(v, tw[n2 * k1]);
            Z[(k1 * P2 + n2) * S] = v;
        });
    }
    // The two twiddled steps with the twiddles in a per-layout table, laid out so that the
    // threads of one step read consecutive entries (no shared-memory bank conflicts; the
    // natural-order table is read with stride k1 or n2 across threads):
    // twA[k1 N2 + n2] = twB[n2 N1 + k1] = W_N^{n2 k1}.  Same values, same results.
    template <int S = 1>
    __host__ __device__ static __forceinline__ void fwd_a_t(float2 (&a)[N1], int n2, float2* Z, const float2* twA) {
        dft<N1, false>(a);
        static_for<0, N1>([&](auto kI) {
            constexpr int k1 = decltype(kI)::value;
            float2 v = a[k1];
            if constexpr (k1 > 0) v = cmul(v, twA[k1 * N2 + n2]);
            Z[(k1 * P2 + n2) * S] = v;
        });
    }
    template <int S = 1>
    __host__ __device__ static __forceinline__ void inv_b_t(float2 (&b)[N2], int k1, float2* Z, const float2* twB) {
        dft<N2, true>(b);
        static_for<0, N2>([&](auto nI) {
            constexpr int n2 = decltype(nI)::value;
            float2 v = b[n2];
            if constexpr (n2 > 0) v = cmulc(v, twB[n2 * N1 + k1]);
            Z[(k1 * P2 + n2) * S] = v;
        });
    }
    // twA and twB (N entries each) from the natural-order table tw; entries i = tid, tid + nthr, ...
    __host__ __device__ static __forceinline__ void fill_tables(float2* twA, float2* twB, const float2* tw, int tid,
                                                                int nthr) {
        for (int i = tid; i < N; i += nthr) {
            const int ka = i / N2, na = i - ka * N2;
            twA[i] = tw[na * ka];
            const int nb = i / N1, kb = i - nb * N1;
            twB[i] = tw[nb * kb];
        }
    }

    // inverse, A layout: a[k1] = Z[k1 P2 + n2] -> inverse DFT_N1 -> a[n1] = x[n2 + N2 n1]
    template <int S = 1>
    __host__ __device__ static __forceinline__ void inv_a_load(float2 (&a)[N1], int n2, const float2* Z) {
        static_for<0, N1>([&](auto kI) { a[decltype(kI)::value] = Z[(decltype(kI)::value * P2 + n2) * S]; });
    }
    __host__ __device__ static __forceinline__ void inv_a(float2 (&a)[N1]) { dft<N1, true>(a); }
};


// Three-level register FFT of length N = NA * NM * NB: the length-N2 = NM * NB second stage
// of the two-level split is itself split in two, so that every thread holds at most
// max(NA, NM, NB) values and a sequence is spread over N / min(NA, NM, NB) threads (60 for
// 300 = 5 x 10 x 6 against 20 for the two-level 15 x 20).  With n = N2 n1 + NB n_m + n_b and
// k = k1 + NA k_m + NA NM k_b:
//   A step: thread n2 < N2 holds x[N2 n1 + n2] (n1 < NA), DFT_NA over n1, twiddle W_N^{n2 k1},
//           stores Y[k1][n2];
//   M step: thread (k1, n_b) holds Y[k1][NB n_m + n_b] (n_m < NM), DFT_NM over n_m, twiddle
//           W_{N2}^{n_b k_m}, stores V[k1 + NA k_m][n_b];
//   B step: thread kk = k1 + NA k_m holds V[kk][n_b] (n_b < NB), DFT_NB over n_b, giving
//           X[kk + NA NM k_b] (k_b < NB).
// The A and B layouts are those of Fft2<NA, N2> and Fft2<NA NM, NB>, so the passes address
// global memory the same way; the inverse runs B, M, A with conjugate twiddles (N x the
// inverse DFT, as the two-level transform).  Twiddle tables in shared memory:
// twA[k1 N2 + n2] = W_N^{n2 k1} (N entries), twM[k_m NB + n_b] = W_{N2}^{n_b k_m} (N2 entries).
template <int NA_, int NM_, int NB_>
struct Fft3 {
    static constexpr int NA = NA_, NM = NM_, NB = NB_;
    static constexpr int N = NA * NM * NB;
    static constexpr int N2 = NM * NB;
    static constexpr int kLevels = 3;
    static constexpr int AV = NA, AT = N2, BV = NB, BT = NA * NM, MT = NA * NB;
    static constexpr int T = AT > BT ? (AT > MT ? AT : MT) : (BT > MT ? BT : MT);   // threads per sequence
    // padded rows: Y[k1] rows of PA >= N2 (PA = NB mod 16: the M step's reads of a warp cover
    // consecutive banks), V rows of PB >= NB (odd: the B step's reads are conflict-free)
    static constexpr int PA = N2 + ((NB - N2) % 16 + 16) % 16;
    static constexpr int PB = (NB % 2) ? NB : NB + 1;
    static constexpr int ZS = (NA * PA > BT * PB) ? NA * PA : BT * PB;   // buffer elements per sequence

    __host__ __device__ static __forceinline__ void fill_tables(float2* twA, float2* twM, const float2* tw, int tid,
                                                                int nthr) {
        for (int i = tid; i < N; i += nthr) {
            const int k1 = i / N2, n2 = i - k1 * N2;
            twA[i] = tw[n2 * k1];
            if (i < N2) {
                const int km = i / NB, nb = i - km * NB;
                twM[i] = tw[(NA * nb * km) % N];
            }
        }
    }
    // forward A step (thread n2): a[n1] = x[N2 n1 + n2] -> Y[k1][n2]
    template <int S = 1>
    __host__ __device__ static __forceinline__ void fwd_a_t(float2 (&a)[NA], int n2, float2* Z, const float2* twA) {
        dft<NA, false>(a);
        static_for<0, NA>([&](auto kI) {
            constexpr int k1 = decltype(kI)::value;
            float2 v = a[k1];
            if constexpr (k1 > 0) v = cmul(v, twA[k1 * N2 + n2]);
            Z[(k1 * PA + n2) * S] = v;
        });
    }
    // forward M step (thread t = k1 NB + n_b < MT): Y (in Zi) -> V (in Zo)
    template <int S = 1>
    __host__ __device__ static __forceinline__ void fwd_m(int t, const float2* Zi, float2* Zo, const float2* twM) {
        const int k1 = t / NB, nb = t - k1 * NB;
        float2 u[NM];
        static_for<0, NM>([&](auto mI) {
            constexpr int nm = decltype(mI)::value;
            u[nm] = Zi[(k1 * PA + NB * nm + nb) * S];
        });
        dft<NM, false>(u);
        static_for<0, NM>([&](auto kI) {
            constexpr int km = decltype(kI)::value;
            float2 v = u[km];
            if constexpr (km > 0) v = cmul(v, twM[km * NB + nb]);
            Zo[((k1 + NA * km) * PB + nb) * S] = v;
        });
    }
    // forward B step (thread kk < BT): b[n_b] = V[kk][n_b] -> b[k_b] = X[kk + BT k_b]
    template <int S = 1>
    __host__ __device__ static __forceinline__ void fwd_b_load(float2 (&b)[NB], int kk, const float2* Z) {
        static_for<0, NB>([&](auto nI) { b[decltype(nI)::value] = Z[(kk * PB + decltype(nI)::value) * S]; });
    }
    __host__ __device__ static __forceinline__ void fwd_b(float2 (&b)[NB]) { dft<NB, false>(b); }
    // inverse B step (thread kk): b[k_b] = X[kk + BT k_b] -> V[kk][n_b]
    template <int S = 1>
    __host__ __device__ static __forceinline__ void inv_b_t(float2 (&b)[NB], int kk, float2* Z, const float2* twM) {
        dft<NB, true>(b);
        const int km = kk / NA;
        static_for<0, NB>([&](auto nI) {
            constexpr int nb = decltype(nI)::value;
            float2 v = b[nb];
            if constexpr (nb > 0) v = cmulc(v, twM[km * NB + nb]);
            Z[(kk * PB + nb) * S] = v;
        });
    }
    // inverse M step (thread t = k1 NB + n_b < MT): V (in Zi) -> Y (in Zo)
    template <int S = 1>
    __host__ __device__ static __forceinline__ void inv_m(int t, const float2* Zi, float2* Zo, const float2* twA) {
        const int k1 = t / NB, nb = t - k1 * NB;
        float2 u[NM];
        static_for<0, NM>([&](auto kI) {
            constexpr int km = decltype(kI)::value;
            u[km] = Zi[((k1 + NA * km) * PB + nb) * S];
        });
        dft<NM, true>(u);
        static_for<0, NM>([&](auto mI) {
            constexpr int nm = decltype(mI)::value;
            const int n2 = NB * nm + nb;
            float2 v = u[nm];
            if (k1 > 0) v = cmulc(v, twA[k1 * N2 + n2]);
            Zo[(k1 * PA + n2) * S] = v;
        });
    }
    // inverse A step (thread n2): a[k1] = Y[k1][n2] -> a[n1] = x[N2 n1 + n2]
    template <int S = 1>
    __host__ __device__ static __forceinline__ void inv_a_load(float2 (&a)[NA], int n2, const float2* Z) {
        static_for<0, NA>([&](auto kI) { a[decltype(kI)::value] = Z[(decltype(kI)::value * PA + n2) * S]; });
    }
    __host__ __device__ static __forceinline__ void inv_a(float2 (&a)[NA]) { dft<NA, true>(a); }
};

}  // namespace pat

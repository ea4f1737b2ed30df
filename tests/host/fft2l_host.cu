// Host-side check of the register FFT building blocks used by the fixed-size
// row and column passes (two- and three-level Cooley-Tukey transforms of fft2l.cuh).
// Every function exercised here is __host__ __device__, so the same code that
// runs in the kernels runs on the CPU; no CUDA call is made.
//
// Input (binary, little-endian) on stdin: int32 count, then per case
// int32 N1, int32 N2, int32 N3, float32 x[2 N] (interleaved re, im); N3 = 0 selects the
// two-level transform N = N1 N2, otherwise the three-level N = N1 N2 N3 (A, M, B steps).
// Output on stdout, per case: float32 X[2 N] (forward DFT through the A and B
// layouts), float32 y[2 N] (inverse of X through the B and A layouts, not
// normalised), float32 d[2 N1], float32 e[2 N2] (forward register DFTs of the
// first N1 and N2 samples; three-level: of the first NA and NB samples).
#include <cmath>
#include <cstdio>
#include <cstdint>
#include <cstdlib>
#include <vector>

#include "fft2l.cuh"

using namespace pat;

namespace {

bool read_all(void* p, size_t n) { return std::fread(p, 1, n, stdin) == n; }
void write_all(const void* p, size_t n) { std::fwrite(p, 1, n, stdout); }

template <int N1, int N2>
void run_case(const std::vector<float2>& x) {
    using F = Fft2<N1, N2>;
    constexpr int N = F::N;
    // twiddle table exp(-2 pi i q / N), q < N, as the plan builds it (FP64, stored FP32)
    std::vector<float2> tw(N);
    for (int q = 0; q < N; ++q) {
        const double a = -2.0 * 3.14159265358979323846 * double(q) / double(N);
        tw[q] = make_float2(float(std::cos(a)), float(std::sin(a)));
    }
    std::vector<float2> Z(F::ZS), X(N), y(N);
    // forward: A layout (thread n2 holds x[N2 n1 + n2]) -> transpose -> B layout
    for (int n2 = 0; n2 < N2; ++n2) {
        float2 a[N1];
        for (int n1 = 0; n1 < N1; ++n1) a[n1] = x[N2 * n1 + n2];
        F::fwd_a(a, n2, Z.data(), tw.data());
    }
    for (int k1 = 0; k1 < N1; ++k1) {
        float2 b[N2];
        F::fwd_b_load(b, k1, Z.data());
        F::fwd_b(b);
        for (int k2 = 0; k2 < N2; ++k2) X[k1 + N1 * k2] = b[k2];
    }
    // inverse: B layout (thread k1 holds X[k1 + N1 k2]) -> transpose -> A layout
    for (int k1 = 0; k1 < N1; ++k1) {
        float2 b[N2];
        for (int k2 = 0; k2 < N2; ++k2) b[k2] = X[k1 + N1 * k2];
        F::inv_b(b, k1, Z.data(), tw.data());
    }
    for (int n2 = 0; n2 < N2; ++n2) {
        float2 a[N1];
        F::inv_a_load(a, n2, Z.data());
        F::inv_a(a);
        for (int n1 = 0; n1 < N1; ++n1) y[n2 + N2 * n1] = a[n1];
    }
    // the same transforms with the per-layout twiddle tables of the row passes: bitwise equal
    {
        std::vector<float2> twA(N), twB(N), Z2(F::ZS), X2(N), y2(N);
        F::fill_tables(twA.data(), twB.data(), tw.data(), 0, 1);
        for (int n2 = 0; n2 < N2; ++n2) {
            float2 a[N1];
            for (int n1 = 0; n1 < N1; ++n1) a[n1] = x[N2 * n1 + n2];
            F::fwd_a_t(a, n2, Z2.data(), twA.data());
        }
        for (int k1 = 0; k1 < N1; ++k1) {
            float2 b[N2];
            F::fwd_b_load(b, k1, Z2.data());
            F::fwd_b(b);
            for (int k2 = 0; k2 < N2; ++k2) X2[k1 + N1 * k2] = b[k2];
        }
        for (int k1 = 0; k1 < N1; ++k1) {
            float2 b[N2];
            for (int k2 = 0; k2 < N2; ++k2) b[k2] = X[k1 + N1 * k2];
            F::inv_b_t(b, k1, Z2.data(), twB.data());
        }
        for (int n2 = 0; n2 < N2; ++n2) {
            float2 a[N1];
            F::inv_a_load(a, n2, Z2.data());
            F::inv_a(a);
            for (int n1 = 0; n1 < N1; ++n1) y2[n2 + N2 * n1] = a[n1];
        }
        for (int i = 0; i < N; ++i)
            if (X2[i].x != X[i].x || X2[i].y != X[i].y || y2[i].x != y[i].x || y2[i].y != y[i].y) {
                std::fprintf(stderr, "table-order twiddles differ at %d (N1=%d N2=%d)\n", i, N1, N2);
                std::exit(3);
            }
    }
    float2 d[N1], e[N2];
    for (int i = 0; i < N1; ++i) d[i] = x[i];
    for (int i = 0; i < N2; ++i) e[i] = x[i];
    dft<N1, false>(d);
    dft<N2, false>(e);
    write_all(X.data(), N * sizeof(float2));
    write_all(y.data(), N * sizeof(float2));
    write_all(d, sizeof(d));
    write_all(e, sizeof(e));
}


// three-level: A step (thread n2), M step (thread k1 NB + n_b), B step (thread kk)
template <int NA, int NM, int NB>
void run_case3(const std::vector<float2>& x) {
    using F = Fft3<NA, NM, NB>;
    constexpr int N = F::N, N2 = F::N2;
    std::vector<float2> tw(N);
    for (int q = 0; q < N; ++q) {
        const double a = -2.0 * 3.14159265358979323846 * double(q) / double(N);
        tw[q] = make_float2(float(std::cos(a)), float(std::sin(a)));
    }
    std::vector<float2> twA(N), twM(N2), Z0(F::ZS), Z1(F::ZS), X(N), y(N);
    F::fill_tables(twA.data(), twM.data(), tw.data(), 0, 1);
    for (int n2 = 0; n2 < N2; ++n2) {
        float2 a[NA];
        for (int n1 = 0; n1 < NA; ++n1) a[n1] = x[N2 * n1 + n2];
        F::fwd_a_t(a, n2, Z0.data(), twA.data());
    }
    for (int t = 0; t < F::MT; ++t) F::fwd_m(t, Z0.data(), Z1.data(), twM.data());
    for (int kk = 0; kk < F::BT; ++kk) {
        float2 b[NB];
        F::fwd_b_load(b, kk, Z1.data());
        F::fwd_b(b);
        for (int kb = 0; kb < NB; ++kb) X[kk + F::BT * kb] = b[kb];
    }
    for (int kk = 0; kk < F::BT; ++kk) {
        float2 b[NB];
        for (int kb = 0; kb < NB; ++kb) b[kb] = X[kk + F::BT * kb];
        F::inv_b_t(b, kk, Z0.data(), twM.data());
    }
    for (int t = 0; t < F::MT; ++t) F::inv_m(t, Z0.data(), Z1.data(), twA.data());
    for (int n2 = 0; n2 < N2; ++n2) {
        float2 a[NA];
        F::inv_a_load(a, n2, Z1.data());
        F::inv_a(a);
        for (int n1 = 0; n1 < NA; ++n1) y[n2 + N2 * n1] = a[n1];
    }
    float2 d[NA], e[NB];
    for (int i = 0; i < NA; ++i) d[i] = x[i];
    for (int i = 0; i < NB; ++i) e[i] = x[i];
    dft<NA, false>(d);
    dft<NB, false>(e);
    write_all(X.data(), N * sizeof(float2));
    write_all(y.data(), N * sizeof(float2));
    write_all(d, sizeof(d));
    write_all(e, sizeof(e));
}

template <int NA, int NM, int NB>
bool dispatch_three(int a, int m, int b, const std::vector<float2>& x) {
    if (a != NA || m != NM || b != NB) return false;
    run_case3<NA, NM, NB>(x);
    return true;
}

bool dispatch3(int a, int m, int b, const std::vector<float2>& x) {
    return dispatch_three<5, 10, 6>(a, m, b, x) || dispatch_three<5, 12, 5>(a, m, b, x) ||
           dispatch_three<5, 6, 10>(a, m, b, x) || dispatch_three<4, 3, 9>(a, m, b, x) ||
           dispatch_three<3, 4, 5>(a, m, b, x) || dispatch_three<2, 3, 2>(a, m, b, x);
}

// the factorisations of the compiled grid sides (both orders)
template <int N1, int N2>
bool dispatch_one(int n1, int n2, const std::vector<float2>& x) {
    if (n1 != N1 || n2 != N2) return false;
    run_case<N1, N2>(x);
    return true;
}

bool dispatch(int n1, int n2, const std::vector<float2>& x) {
    return dispatch_one<12, 9>(n1, n2, x) || dispatch_one<9, 12>(n1, n2, x) || dispatch_one<12, 12>(n1, n2, x) ||
           dispatch_one<12, 15>(n1, n2, x) || dispatch_one<15, 12>(n1, n2, x) ||
           dispatch_one<20, 10>(n1, n2, x) || dispatch_one<10, 20>(n1, n2, x) ||
           dispatch_one<16, 15>(n1, n2, x) || dispatch_one<15, 16>(n1, n2, x) ||
           dispatch_one<20, 15>(n1, n2, x) || dispatch_one<15, 20>(n1, n2, x) ||
           dispatch_one<2, 3>(n1, n2, x) || dispatch_one<4, 5>(n1, n2, x) || dispatch_one<8, 25>(n1, n2, x);
}

}  // namespace

int main() {
    int32_t count = 0;
    if (!read_all(&count, sizeof(count))) return 2;
    for (int c = 0; c < count; ++c) {
        int32_t nn[3];
        if (!read_all(nn, sizeof(nn))) return 2;
        std::vector<float2> x(size_t(nn[0]) * nn[1] * (nn[2] ? nn[2] : 1));
        if (!read_all(x.data(), x.size() * sizeof(float2))) return 2;
        const bool ok = nn[2] ? dispatch3(nn[0], nn[1], nn[2], x) : dispatch(nn[0], nn[1], x);
        if (!ok) {
            std::fprintf(stderr, "no factorisation %d x %d x %d compiled in\n", nn[0], nn[1], nn[2]);
            return 3;
        }
    }
    std::fflush(stdout);
    return 0;
}

// Batched complex FFTs of 5-smooth length in shared memory (Stockham
// auto-sort, radix 2/3/4/5), used by the row and column passes of the
// k-space time stepping.  Twiddles come from a table exp(-2 pi i q / n),
// q < n, built in FP64 on the host and staged in shared memory.
#pragma once

#include <cuda_runtime.h>

namespace pat {

constexpr int kMaxStages = 12;

// Radix schedule of one FFT length: n = rad[0] * rad[1] * ... * rad[nrad-1].
struct FftDesc {
    int n;
    int nrad;
    int rad[kMaxStages];
};

__host__ __device__ __forceinline__ float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__host__ __device__ __forceinline__ float2 csub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
__host__ __device__ __forceinline__ float2 cmul(float2 a, float2 b) {
    return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
// a * conj(b)
__host__ __device__ __forceinline__ float2 cmulc(float2 a, float2 b) {
    return make_float2(a.x * b.x + a.y * b.y, a.y * b.x - a.x * b.y);
}
__host__ __device__ __forceinline__ float2 cscale(float2 a, float s) { return make_float2(a.x * s, a.y * s); }
// multiply by -i (forward) or +i (inverse)
template <bool INV>
__host__ __device__ __forceinline__ float2 rot(float2 a) {
    return INV ? make_float2(-a.y, a.x) : make_float2(a.y, -a.x);
}

// In-register DFT of R points: v_q <- sum_m v_m exp(-+ 2 pi i m q / R).
template <int R, bool INV>
__host__ __device__ __forceinline__ void dft_small(float2 (&v)[R]) {
    if constexpr (R == 2) {
        float2 a = v[0], b = v[1];
        v[0] = cadd(a, b);
        v[1] = csub(a, b);
    } else if constexpr (R == 3) {
        const float s3 = 0.86602540378443864676f;   // sin(2 pi / 3)
        float2 sum = cadd(v[1], v[2]);
        float2 dif = csub(v[1], v[2]);
        float2 m = make_float2(v[0].x - 0.5f * sum.x, v[0].y - 0.5f * sum.y);
        float2 t = rot<INV>(cscale(dif, s3));
        v[0] = cadd(v[0], sum);
        v[1] = cadd(m, t);
        v[2] = csub(m, t);
    } else if constexpr (R == 4) {
        float2 a = cadd(v[0], v[2]), b = csub(v[0], v[2]);
        float2 c = cadd(v[1], v[3]), d = rot<INV>(csub(v[1], v[3]));
        v[0] = cadd(a, c);
        v[2] = csub(a, c);
        v[1] = cadd(b, d);
        v[3] = csub(b, d);
    } else if constexpr (R == 5) {
        const float c1 = 0.30901699437494742410f;    // cos(2 pi / 5)
        const float c2 = -0.80901699437494742410f;   // cos(4 pi / 5)
        const float s1 = 0.95105651629515357212f;    // sin(2 pi / 5)
        const float s2 = 0.58778525229247312917f;    // sin(4 pi / 5)
        float2 a1 = cadd(v[1], v[4]), b1 = csub(v[1], v[4]);
        float2 a2 = cadd(v[2], v[3]), b2 = csub(v[2], v[3]);
        float2 m1 = make_float2(v[0].x + c1 * a1.x + c2 * a2.x, v[0].y + c1 * a1.y + c2 * a2.y);
        float2 m2 = make_float2(v[0].x + c2 * a1.x + c1 * a2.x, v[0].y + c2 * a1.y + c1 * a2.y);
        float2 t1 = rot<INV>(make_float2(s1 * b1.x + s2 * b2.x, s1 * b1.y + s2 * b2.y));
        float2 t2 = rot<INV>(make_float2(s2 * b1.x - s1 * b2.x, s2 * b1.y - s1 * b2.y));
        v[0] = make_float2(v[0].x + a1.x + a2.x, v[0].y + a1.y + a2.y);
        v[1] = cadd(m1, t1);
        v[4] = csub(m1, t1);
        v[2] = cadd(m2, t2);
        v[3] = csub(m2, t2);
    }
}

// One Stockham stage of radix R over nseq sequences (stride ss) from src to dst.
// Ns is the length of the sub-transforms already done.
template <int R, bool INV>
__device__ __forceinline__ void stockham_stage(const float2* __restrict__ src, float2* __restrict__ dst,
                                               int n, int Ns, int nseq, int ss,
                                               const float2* __restrict__ tw) {
    const int nb = n / R;
    const int tstride = n / (Ns * R);
    const int total = nseq * nb;
    for (int t = threadIdx.x; t < total; t += blockDim.x) {
        const int s = t / nb;
        const int j = t - s * nb;
        const float2* in = src + s * ss;
        float2* out = dst + s * ss;
        const int k = j % Ns;
        float2 v[R];
#pragma unroll
        for (int r = 0; r < R; ++r) v[r] = in[j + r * nb];
        if (Ns > 1) {
#pragma unroll
            for (int r = 1; r < R; ++r) {
                const float2 w = tw[r * k * tstride];
                v[r] = INV ? cmulc(v[r], w) : cmul(v[r], w);
            }
        }
        dft_small<R, INV>(v);
        const int base = (j - k) * R + k;
#pragma unroll
        for (int r = 0; r < R; ++r) out[base + r * Ns] = v[r];
    }
}

// FFT of nseq sequences of length fd.n held at a[s*ss + i]; b is scratch of
// the same shape.  Unnormalised; INV selects exp(+2 pi i ...).  All threads
// of the block must call it; it ends with __syncthreads().  Returns the
// buffer (a or b) that holds the result.
template <bool INV>
__device__ float2* fft_smem(float2* a, float2* b, int nseq, int ss, const FftDesc& fd,
                            const float2* __restrict__ tw) {
    int Ns = 1;
    for (int st = 0; st < fd.nrad; ++st) {
        const int R = fd.rad[st];
        switch (R) {
            case 2: stockham_stage<2, INV>(a, b, fd.n, Ns, nseq, ss, tw); break;
            case 3: stockham_stage<3, INV>(a, b, fd.n, Ns, nseq, ss, tw); break;
            case 4: stockham_stage<4, INV>(a, b, fd.n, Ns, nseq, ss, tw); break;
            default: stockham_stage<5, INV>(a, b, fd.n, Ns, nseq, ss, tw); break;
        }
        __syncthreads();
        float2* t = a;
        a = b;
        b = t;
        Ns *= R;
    }
    return a;
}

}  // namespace pat

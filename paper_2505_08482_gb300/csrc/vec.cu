// Vector kernels of the optimiser and the multigrid schedule: FP64-accumulated
// dot products (deterministic two-stage reduction), device-scalar axpy for the
// two-loop recursion, block scaling, projection onto the box, direction
// clipping, bilinear resampling between levels and linear time interpolation
// of the data.
#include <cuda_runtime.h>

#include "pat_internal.h"
#include "vec.h"

namespace pat {

__global__ void __launch_bounds__(256) k_dot_partial(const float* __restrict__ a, const float* __restrict__ b,
                                                     size_t n, double* __restrict__ part) {
    __shared__ double red[256];
    double acc = 0.0;
    for (size_t i = size_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += size_t(gridDim.x) * blockDim.x)
        acc += double(a[i]) * double(b[i]);
    red[threadIdx.x] = acc;
    __syncthreads();
    for (int s = 128; s > 0; s >>= 1) {
        if (threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
        __syncthreads();
    }
    if (threadIdx.x == 0) part[blockIdx.x] = red[0];
}

// out = mul * (sum of partials) [* (*scale) if scale]
__global__ void k_dot_final(const double* __restrict__ part, int np, double* __restrict__ out,
                            const double* __restrict__ scale, double mul) {
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        double s = 0.0;
        for (int i = 0; i < np; ++i) s += part[i];
        s *= mul;
        if (scale) s *= *scale;
        *out = s;
    }
}

// y += sign * (coef[0] - (coef2 ? coef2[0] : 0)) * x
__global__ void k_axpy_dev(float* __restrict__ y, const float* __restrict__ x, size_t n,
                           const double* __restrict__ coef, const double* __restrict__ coef2, float sign) {
    const double cv = coef[0] - (coef2 ? coef2[0] : 0.0);
    const float c = sign * float(cv);
    for (size_t i = size_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += size_t(gridDim.x) * blockDim.x)
        y[i] += c * x[i];
}

__global__ void k_scale_dev(float* __restrict__ y, const float* __restrict__ x, size_t n,
                            const double* __restrict__ coef, float sign) {
    const float c = sign * float(coef[0]);
    for (size_t i = size_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += size_t(gridDim.x) * blockDim.x)
        y[i] = c * x[i];
}

__global__ void k_axpby(float* __restrict__ out, float a, const float* __restrict__ x, float b,
                        const float* __restrict__ y, size_t n) {
    for (size_t i = size_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += size_t(gridDim.x) * blockDim.x)
        out[i] = a * x[i] + (y ? b * y[i] : 0.f);
}

__global__ void k_fill(float* __restrict__ y, float v, size_t n) {
    for (size_t i = size_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += size_t(gridDim.x) * blockDim.x)
        y[i] = v;
}

// out[i] = v[i] * s_b or / s_b with s_b = s0 for i < n0 and s1 otherwise
__global__ void k_blockscale(float* __restrict__ out, const float* __restrict__ v, size_t n, size_t n0, float s0,
                             float s1, int divide) {
    for (size_t i = size_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += size_t(gridDim.x) * blockDim.x) {
        const float s = i < n0 ? s0 : s1;
        out[i] = divide ? v[i] / s : v[i] * s;
    }
}

// z_t = clamp(z + alpha d, lo, hi), x_t = sigma z_t  (bounds per block)
__global__ void k_project(float* __restrict__ zt, float* __restrict__ xt, const float* __restrict__ z,
                          const float* __restrict__ d, float alpha, size_t n, size_t n0, Box box) {
    for (size_t i = size_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += size_t(gridDim.x) * blockDim.x) {
        const bool p = i < n0;
        const float lo = p ? box.lo0 : box.lo1, hi = p ? box.hi0 : box.hi1, s = p ? box.s0 : box.s1;
        const float v = fminf(fmaxf(z[i] + alpha * d[i], lo), hi);
        zt[i] = v;
        xt[i] = v * s;
    }
}

// zero the components of d that leave the box at variables already on a bound
__global__ void k_clip_dir(float* __restrict__ d, const float* __restrict__ z, size_t n, size_t n0, Box box) {
    for (size_t i = size_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += size_t(gridDim.x) * blockDim.x) {
        const bool p = i < n0;
        const float lo = p ? box.lo0 : box.lo1, hi = p ? box.hi0 : box.hi1;
        if ((z[i] <= lo && d[i] < 0.f) || (z[i] >= hi && d[i] > 0.f)) d[i] = 0.f;
    }
}

__global__ void k_absmax_partial(const float* __restrict__ a, size_t n, double* __restrict__ part) {
    __shared__ float red[256];
    float m = 0.f;
    for (size_t i = size_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += size_t(gridDim.x) * blockDim.x)
        m = fmaxf(m, fabsf(a[i]));
    red[threadIdx.x] = m;
    __syncthreads();
    for (int s = 128; s > 0; s >>= 1) {
        if (threadIdx.x < s) red[threadIdx.x] = fmaxf(red[threadIdx.x], red[threadIdx.x + s]);
        __syncthreads();
    }
    if (threadIdx.x == 0) part[blockIdx.x] = red[0];
}

__global__ void k_max_final(const double* __restrict__ part, int np, double* __restrict__ out) {
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        double m = 0.0;
        for (int i = 0; i < np; ++i) m = fmax(m, part[i]);
        *out = m;
    }
}

// bilinear resampling of nb fields [nb][ns][ns] -> [nb][nd][nd] on cell-centred
// coordinates of the same physical square, constant beyond the outer centres
__global__ void k_resample(const float* __restrict__ src, float* __restrict__ dst, int nb, int ns, int nd) {
    const size_t total = size_t(nb) * nd * nd;
    const double ratio = double(ns) / double(nd);
    for (size_t i = size_t(blockIdx.x) * blockDim.x + threadIdx.x; i < total; i += size_t(gridDim.x) * blockDim.x) {
        const int b = int(i / (size_t(nd) * nd));
        const int rem = int(i - size_t(b) * nd * nd);
        const int iy = rem / nd, ix = rem - iy * nd;
        double u = (ix + 0.5) * ratio - 0.5, v = (iy + 0.5) * ratio - 0.5;
        u = fmin(fmax(u, 0.0), ns - 1.0);
        v = fmin(fmax(v, 0.0), ns - 1.0);
        int x0 = int(floor(u)), y0 = int(floor(v));
        x0 = min(x0, max(ns - 2, 0));
        y0 = min(y0, max(ns - 2, 0));
        const int x1 = min(x0 + 1, ns - 1), y1 = min(y0 + 1, ns - 1);
        const float fx = float(u - x0), fy = float(v - y0);
        const float* s = src + size_t(b) * ns * ns;
        const float top = s[size_t(y0) * ns + x0] * (1.f - fx) + s[size_t(y0) * ns + x1] * fx;
        const float bot = s[size_t(y1) * ns + x0] * (1.f - fx) + s[size_t(y1) * ns + x1] * fx;
        dst[i] = top * (1.f - fy) + bot * fy;
    }
}

// linear interpolation in time of y[K][nts][m] (t = n dts) to t = n dtd, n < ntd
__global__ void k_time_interp(const float* __restrict__ y, float* __restrict__ out, int K, int nts, int ntd, int m,
                              double dts, double dtd) {
    const size_t total = size_t(K) * ntd * m;
    for (size_t i = size_t(blockIdx.x) * blockDim.x + threadIdx.x; i < total; i += size_t(gridDim.x) * blockDim.x) {
        const int k = int(i / (size_t(ntd) * m));
        const int rem = int(i - size_t(k) * ntd * m);
        const int n = rem / m, s = rem - n * m;
        const float* yk = y + size_t(k) * nts * m;
        const double u = n * dtd / dts;
        float v;
        if (u >= nts - 1) {
            v = yk[size_t(nts - 1) * m + s];
        } else {
            const int i0 = int(floor(u));
            const float f = float(u - i0);
            v = yk[size_t(i0) * m + s] * (1.f - f) + yk[size_t(i0 + 1) * m + s] * f;
        }
        out[i] = v;
    }
}

// ---- launchers ----
static unsigned blocks_for(size_t n) {
    size_t b = (n + 255) / 256;
    return unsigned(b < 1 ? 1 : (b > 2048 ? 2048 : b));
}

static int chk(const char* w) {
    count_launch();
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? PAT_OK : cuda_fail(e, w);
}

int vdot(cudaStream_t st, const float* a, const float* b, size_t n, double* out, double* part,
         const double* scale, double mul) {
    count_launch();
    k_dot_partial<<<kPartials, 256, 0, st>>>(a, b, n, part);
    k_dot_final<<<1, 32, 0, st>>>(part, kPartials, out, scale, mul);
    return chk("vdot");
}

int vaxpy_dev(cudaStream_t st, float* y, const float* x, size_t n, const double* coef, const double* coef2,
              float sign) {
    k_axpy_dev<<<blocks_for(n), 256, 0, st>>>(y, x, n, coef, coef2, sign);
    return chk("vaxpy_dev");
}

int vscale_dev(cudaStream_t st, float* y, const float* x, size_t n, const double* coef, float sign) {
    k_scale_dev<<<blocks_for(n), 256, 0, st>>>(y, x, n, coef, sign);
    return chk("vscale_dev");
}

int vaxpby(cudaStream_t st, float* out, float a, const float* x, float b, const float* y, size_t n) {
    k_axpby<<<blocks_for(n), 256, 0, st>>>(out, a, x, b, y, n);
    return chk("vaxpby");
}

int vfill(cudaStream_t st, float* y, float v, size_t n) {
    k_fill<<<blocks_for(n), 256, 0, st>>>(y, v, n);
    return chk("vfill");
}

int vblockscale(cudaStream_t st, float* out, const float* v, size_t n, size_t n0, float s0, float s1, int divide) {
    k_blockscale<<<blocks_for(n), 256, 0, st>>>(out, v, n, n0, s0, s1, divide);
    return chk("vblockscale");
}

int vproject(cudaStream_t st, float* zt, float* xt, const float* z, const float* d, float alpha, size_t n,
             size_t n0, const Box& box) {
    k_project<<<blocks_for(n), 256, 0, st>>>(zt, xt, z, d, alpha, n, n0, box);
    return chk("vproject");
}

int vclip_dir(cudaStream_t st, float* d, const float* z, size_t n, size_t n0, const Box& box) {
    k_clip_dir<<<blocks_for(n), 256, 0, st>>>(d, z, n, n0, box);
    return chk("vclip_dir");
}

int vabsmax(cudaStream_t st, const float* a, size_t n, double* out, double* part) {
    count_launch();
    k_absmax_partial<<<kPartials, 256, 0, st>>>(a, n, part);
    k_max_final<<<1, 32, 0, st>>>(part, kPartials, out);
    return chk("vabsmax");
}

int vresample(cudaStream_t st, const float* src, float* dst, int nb, int ns, int nd) {
    k_resample<<<blocks_for(size_t(nb) * nd * nd), 256, 0, st>>>(src, dst, nb, ns, nd);
    return chk("vresample");
}

int vtime_interp(cudaStream_t st, const float* y, float* out, int K, int nts, int ntd, int m, double dts,
                 double dtd) {
    k_time_interp<<<blocks_for(size_t(K) * ntd * m), 256, 0, st>>>(y, out, K, nts, ntd, m, dts, dtd);
    return chk("vtime_interp");
}

}  // namespace pat

// ---- C ABI of the two multigrid transfers (Sec. 3.1, Sec. 4.1.2) ----

extern "C" int pat_prolong(const float* d_src, float* d_dst, int nb, int n_src, int n_dst, void* stream) {
    if (!d_src || !d_dst || nb < 1 || n_src < 1 || n_dst < 1) {
        pat::set_error("pat_prolong: null buffer or size < 1");
        return PAT_EINVAL;
    }
    return pat::vresample(static_cast<cudaStream_t>(stream), d_src, d_dst, nb, n_src, n_dst);
}

extern "C" int pat_time_interp(const float* d_y, float* d_out, int K, int nt_src, int nt_dst, int m, double dt_src,
                               double dt_dst, void* stream) {
    if (!d_y || !d_out || K < 1 || nt_src < 1 || nt_dst < 1 || m < 1 || !(dt_src > 0.0) || !(dt_dst > 0.0)) {
        pat::set_error("pat_time_interp: null buffer, size < 1 or time step not positive");
        return PAT_EINVAL;
    }
    return pat::vtime_interp(static_cast<cudaStream_t>(stream), d_y, d_out, K, nt_src, nt_dst, m, dt_src, dt_dst);
}

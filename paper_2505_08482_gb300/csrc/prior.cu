// Ornstein-Uhlenbeck prior terms of the objective (Eq. Minimised_functional,
// Sec. 4.1.2): for a field z on the n x n grid, P(z) = 1/2 (z - eta)^T
// Xi^{-1} (z - eta) / sigma^2 and dP/dz = Xi^{-1} (z - eta) / sigma^2 with
// Xi_ij = exp(-|r_i - r_j| / tau).
//
// Xi v is a linear convolution of v with the kernel exp(-|r| / tau) over the
// offsets (-n, n)^2.  On a torus of side M >= 2n - 1 (5-smooth) the periodic
// kernel k defines a circulant C with Xi = P^T C P (P: zero-padding of the
// n x n field), and C = F^-1 diag(lambda) F with lambda = FFT2(k) real (k is
// even).  So Xi v = restrict(IFFT2(lambda FFT2(pad v))), exactly.  Xi^{-1} b
// is found by preconditioned conjugate gradients with the preconditioner
// P^T C^{-1} P (same transforms, 1/lambda), batched over fields with per-field
// FP64 scalars.  lambda is computed on the host in FP64 as C_M k C_M (k even:
// the 2-D DFT is a cosine transform) and stored in FP32.
//
// Two real fields share one complex transform (re, im): lambda is real and
// even, so the product keeps them apart.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <new>
#include <vector>

#include "pat_internal.h"

using namespace pat;

struct pat_prior_s {
    int n, M, maxf, device;
    double dx, tau;
    FftDesc fd;
    float2* tw = nullptr;     // [M] exp(-2 pi i q / M)
    float* lam = nullptr;     // [M][M] spectrum of the circulant embedding
    float* ilam = nullptr;    // [M][M] 1 / lambda (preconditioner)
    float2* W = nullptr;      // [(maxf+1)/2][M][M] transform work
    float* b = nullptr;       // [maxf][n][n] right-hand side
    float* r = nullptr;       // residual
    float* s = nullptr;       // preconditioned residual
    float* d = nullptr;       // search direction
    float* q = nullptr;       // Xi d
    double* part = nullptr;   // [maxf][kDotBlocks] dot partials
    double* sc = nullptr;     // [kSc][maxf] per-field scalars
    int* active = nullptr;    // [maxf] field not yet converged
    int* nactive = nullptr;   // [1]
    int rows_per_cta, cols_per_cta;
    size_t smem_rows, smem_cols;
};

namespace {

constexpr int kDotBlocks = 64;
enum { SC_RS = 0, SC_BB, SC_ALPHA, SC_BETA, SC_ETA, SC_COEF, SC_ISIG2, kSc };

// ---- transforms ----------------------------------------------------------
// rows y < n of the padded fields (2p, 2p+1) -> row FFT -> W[p][y][:]
__global__ void k_pr_rows_fwd(const float* __restrict__ v, float2* __restrict__ W, int n, int M, int nf, FftDesc fd,
                              const float2* __restrict__ twg, int R) {
    extern __shared__ float2 sm[];
    float2* tw = sm;
    float2* a = tw + M;
    float2* b = a + R * M;
    const int p = blockIdx.y, y0 = blockIdx.x * R;
    const int nr = min(R, n - y0);
    for (int i = threadIdx.x; i < M; i += blockDim.x) tw[i] = twg[i];
    const size_t nn = size_t(n) * n;
    const float* va = v + size_t(2 * p) * nn;
    const float* vb = (2 * p + 1 < nf) ? v + size_t(2 * p + 1) * nn : nullptr;
    for (int i = threadIdx.x; i < R * M; i += blockDim.x) {
        const int rr = i / M, x = i - rr * M;
        float re = 0.f, im = 0.f;
        if (rr < nr && x < n) {
            const size_t o = size_t(y0 + rr) * n + x;
            re = va[o];
            if (vb) im = vb[o];
        }
        a[i] = make_float2(re, im);
    }
    __syncthreads();
    const float2* res = fft_smem<false>(a, b, R, M, fd, tw);
    for (int i = threadIdx.x; i < nr * M; i += blockDim.x) {
        const int rr = i / M, x = i - rr * M;
        W[(size_t(p) * M + y0 + rr) * M + x] = res[i];
    }
}

// columns of W (rows >= n are zero) -> FFT -> times L -> inverse FFT -> rows < n of W.
// The C sequences sit at stride M + 1 in shared memory (no bank conflicts in the transpose).
__global__ void k_pr_cols(float2* __restrict__ W, const float* __restrict__ L, int n, int M, FftDesc fd,
                          const float2* __restrict__ twg, int C) {
    extern __shared__ float2 sm[];
    const int S = M + 1;
    float2* tw = sm;
    float2* a = tw + M;
    float2* b = a + C * S;
    const int p = blockIdx.y, x0 = blockIdx.x * C;
    const int nc = min(C, M - x0);
    for (int i = threadIdx.x; i < M; i += blockDim.x) tw[i] = twg[i];
    float2* Wp = W + size_t(p) * M * M;
    for (int i = threadIdx.x; i < C * M; i += blockDim.x) {
        const int y = i / C, c = i - y * C;
        a[c * S + y] = (y < n && c < nc) ? Wp[size_t(y) * M + x0 + c] : make_float2(0.f, 0.f);
    }
    __syncthreads();
    float2* f = fft_smem<false>(a, b, C, S, fd, tw);
    float2* g = (f == a) ? b : a;
    for (int i = threadIdx.x; i < C * M; i += blockDim.x) {
        const int c = i / M, ky = i - c * M;
        const float l = (c < nc) ? L[size_t(ky) * M + x0 + c] : 0.f;
        f[c * S + ky] = cscale(f[c * S + ky], l);
    }
    __syncthreads();
    const float2* res = fft_smem<true>(f, g, C, S, fd, tw);
    for (int i = threadIdx.x; i < C * n; i += blockDim.x) {
        const int y = i / C, c = i - y * C;
        if (c < nc) Wp[size_t(y) * M + x0 + c] = res[c * S + y];
    }
}

// rows y < n of W -> inverse row FFT -> fields (2p, 2p+1), scaled by 1 / M^2
__global__ void k_pr_rows_inv(const float2* __restrict__ W, float* __restrict__ out, int n, int M, int nf,
                              FftDesc fd, const float2* __restrict__ twg, int R) {
    extern __shared__ float2 sm[];
    float2* tw = sm;
    float2* a = tw + M;
    float2* b = a + R * M;
    const int p = blockIdx.y, y0 = blockIdx.x * R;
    const int nr = min(R, n - y0);
    for (int i = threadIdx.x; i < M; i += blockDim.x) tw[i] = twg[i];
    for (int i = threadIdx.x; i < R * M; i += blockDim.x) {
        const int rr = i / M, x = i - rr * M;
        a[i] = rr < nr ? W[(size_t(p) * M + y0 + rr) * M + x] : make_float2(0.f, 0.f);
    }
    __syncthreads();
    const float2* res = fft_smem<true>(a, b, R, M, fd, tw);
    const size_t nn = size_t(n) * n;
    const float s = 1.f / (float(M) * float(M));
    float* oa = out + size_t(2 * p) * nn;
    float* ob = (2 * p + 1 < nf) ? out + size_t(2 * p + 1) * nn : nullptr;
    for (int i = threadIdx.x; i < nr * n; i += blockDim.x) {
        const int rr = i / n, x = i - rr * n;
        const float2 z = res[rr * M + x];
        const size_t o = size_t(y0 + rr) * n + x;
        oa[o] = s * z.x;
        if (ob) ob[o] = s * z.y;
    }
}

// ---- batched vector kernels over nf fields of nn values ------------------
__global__ void k_pr_dot(const float* __restrict__ a, const float* __restrict__ b, size_t nn,
                         double* __restrict__ part) {
    __shared__ double red[256];
    const int f = blockIdx.y;
    const float* af = a + size_t(f) * nn;
    const float* bf = b + size_t(f) * nn;
    double acc = 0.0;
    for (size_t i = size_t(blockIdx.x) * blockDim.x + threadIdx.x; i < nn; i += size_t(gridDim.x) * blockDim.x)
        acc += double(af[i]) * double(bf[i]);
    red[threadIdx.x] = acc;
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) part[size_t(f) * gridDim.x + blockIdx.x] = red[0];
}

__device__ __forceinline__ double sum_part(const double* part, int f) {
    double s = 0.0;
    for (int j = 0; j < kDotBlocks; ++j) s += part[f * kDotBlocks + j];   // fixed order
    return s;
}

// per-field scalar steps of PCG (one thread per field)
// 0: rs = <r,s>, bb = <b,b> from part[0..nf) and part[nf..2nf); all fields active
// 1: alpha = rs / <d,q>
// 2: active &= <r,r> > tol2 bb; count the active fields
// 3: beta = <r,s>_new / rs, rs = <r,s>_new
// 4: J += sum_f 1/2 <b,z>_f / sigma_f^2 (thread 0, fixed order)
__global__ void k_pr_scalar(int mode, const double* __restrict__ part, double* __restrict__ sc, int* __restrict__ active,
                            int* __restrict__ nactive, int nf, int maxf, double tol2, double* __restrict__ J) {
    const int f = threadIdx.x;
    double* rs = sc + SC_RS * maxf;
    double* bb = sc + SC_BB * maxf;
    double* alpha = sc + SC_ALPHA * maxf;
    double* beta = sc + SC_BETA * maxf;
    if (mode == 4) {
        if (f == 0 && J) {
            double v = 0.0;
            for (int k = 0; k < nf; ++k) v += 0.5 * sum_part(part, k) * sc[SC_ISIG2 * maxf + k];
            *J += v;
        }
        return;
    }
    if (mode == 2 && f == 0) *nactive = 0;
    __syncthreads();
    if (f >= nf) return;
    if (mode == 0) {
        rs[f] = sum_part(part, f);
        bb[f] = sum_part(part + size_t(nf) * kDotBlocks, f);
        active[f] = 1;
    } else if (mode == 1) {
        const double dq = sum_part(part, f);
        alpha[f] = (active[f] && dq > 0.0 && isfinite(dq) && isfinite(rs[f])) ? rs[f] / dq : 0.0;
    } else if (mode == 2) {
        const double rr = sum_part(part, f);
        if (!(rr > tol2 * bb[f]) || !isfinite(rr)) active[f] = 0;
        if (active[f]) atomicAdd(nactive, 1);
    } else if (mode == 3) {
        const double rn = sum_part(part, f);
        beta[f] = (active[f] && rs[f] > 0.0 && isfinite(rn)) ? rn / rs[f] : 0.0;
        rs[f] = rn;
    }
}

// z += alpha d; r -= alpha q
__global__ void k_pr_update(float* __restrict__ z, float* __restrict__ r, const float* __restrict__ d,
                            const float* __restrict__ q, const double* __restrict__ alpha, size_t nn, int nf) {
    const size_t tot = nn * nf;
    for (size_t i = size_t(blockIdx.x) * blockDim.x + threadIdx.x; i < tot; i += size_t(gridDim.x) * blockDim.x) {
        const float a = float(alpha[i / nn]);
        z[i] += a * d[i];
        r[i] -= a * q[i];
    }
}

// d = s + beta d
__global__ void k_pr_dir(float* __restrict__ d, const float* __restrict__ s, const double* __restrict__ beta, size_t nn,
                         int nf) {
    const size_t tot = nn * nf;
    for (size_t i = size_t(blockIdx.x) * blockDim.x + threadIdx.x; i < tot; i += size_t(gridDim.x) * blockDim.x)
        d[i] = s[i] + float(beta[i / nn]) * d[i];
}

// out = a - coef_f b  (coef = eta: right-hand side x - eta; coef = 1: residual b - Xi z)
__global__ void k_pr_axpy(float* __restrict__ out, const float* __restrict__ a, const float* __restrict__ b,
                          const double* __restrict__ coef, float cb, size_t nn, int nf) {
    const size_t tot = nn * nf;
    for (size_t i = size_t(blockIdx.x) * blockDim.x + threadIdx.x; i < tot; i += size_t(gridDim.x) * blockDim.x) {
        const float c = coef ? float(coef[i / nn]) : cb;
        out[i] = a[i] - c * (b ? b[i] : 1.f);
    }
}

// grad += coef_f z
__global__ void k_pr_grad(float* __restrict__ g, const float* __restrict__ z, const double* __restrict__ coef,
                          size_t nn, int nf) {
    const size_t tot = nn * nf;
    for (size_t i = size_t(blockIdx.x) * blockDim.x + threadIdx.x; i < tot; i += size_t(gridDim.x) * blockDim.x)
        g[i] += float(coef[i / nn]) * z[i];
}

unsigned vec_blocks(size_t tot) { return unsigned(std::min<size_t>((tot + 255) / 256, 4096)); }

int chk(const char* what) {
    count_launch();
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? PAT_OK : cuda_fail(e, what);
}

#define RC(x)                          \
    do {                               \
        int rc_ = (x);                 \
        if (rc_ != PAT_OK) return rc_; \
    } while (0)

// out = (lam or 1/lam) applied to v: Xi v (inv = false) or the preconditioner (inv = true)
int conv(pat_prior_s* p, const float* v, float* out, int nf, bool inv, cudaStream_t st) {
    const int np = (nf + 1) / 2;
    const dim3 rg((p->n + p->rows_per_cta - 1) / p->rows_per_cta, np);
    k_pr_rows_fwd<<<rg, 256, p->smem_rows, st>>>(v, p->W, p->n, p->M, nf, p->fd, p->tw, p->rows_per_cta);
    RC(chk("k_pr_rows_fwd"));
    const dim3 cg((p->M + p->cols_per_cta - 1) / p->cols_per_cta, np);
    k_pr_cols<<<cg, 256, p->smem_cols, st>>>(p->W, inv ? p->ilam : p->lam, p->n, p->M, p->fd, p->tw, p->cols_per_cta);
    RC(chk("k_pr_cols"));
    k_pr_rows_inv<<<rg, 256, p->smem_rows, st>>>(p->W, out, p->n, p->M, nf, p->fd, p->tw, p->rows_per_cta);
    return chk("k_pr_rows_inv");
}

int dot(pat_prior_s* p, const float* a, const float* b, int nf, double* part, cudaStream_t st) {
    k_pr_dot<<<dim3(kDotBlocks, nf), 256, 0, st>>>(a, b, size_t(p->n) * p->n, part);
    return chk("k_pr_dot");
}

int scalar(pat_prior_s* p, int mode, int nf, double tol2, double* J, cudaStream_t st) {
    k_pr_scalar<<<1, 32 * ((p->maxf + 31) / 32), 0, st>>>(mode, p->part, p->sc, p->active, p->nactive, nf, p->maxf,
                                                          tol2, J);
    return chk("k_pr_scalar");
}

// PCG for Xi z = b (b in p->b); z warm (its contents are the start) or zero
int pcg(pat_prior_s* p, float* z, int nf, double tol, int maxit, bool warm, int* iters, cudaStream_t st) {
    const size_t nn = size_t(p->n) * p->n, tot = nn * nf;
    if (warm) {
        RC(conv(p, z, p->q, nf, false, st));                        // Xi z
        k_pr_axpy<<<vec_blocks(tot), 256, 0, st>>>(p->r, p->b, p->q, nullptr, 1.f, nn, nf);
        RC(chk("k_pr_axpy"));
    } else {
        PAT_CUDA(cudaMemsetAsync(z, 0, tot * sizeof(float), st));
        PAT_CUDA(cudaMemcpyAsync(p->r, p->b, tot * sizeof(float), cudaMemcpyDeviceToDevice, st));
    }
    RC(conv(p, p->r, p->s, nf, true, st));
    PAT_CUDA(cudaMemcpyAsync(p->d, p->s, tot * sizeof(float), cudaMemcpyDeviceToDevice, st));
    RC(dot(p, p->r, p->s, nf, p->part, st));
    RC(dot(p, p->b, p->b, nf, p->part + size_t(nf) * kDotBlocks, st));
    RC(scalar(p, 0, nf, 0.0, nullptr, st));
    const double tol2 = tol * tol;
    int it = 0;
    for (; it < maxit; ++it) {
        RC(conv(p, p->d, p->q, nf, false, st));
        RC(dot(p, p->d, p->q, nf, p->part, st));
        RC(scalar(p, 1, nf, 0.0, nullptr, st));
        k_pr_update<<<vec_blocks(tot), 256, 0, st>>>(z, p->r, p->d, p->q, p->sc + SC_ALPHA * p->maxf, nn, nf);
        RC(chk("k_pr_update"));
        RC(dot(p, p->r, p->r, nf, p->part, st));
        RC(scalar(p, 2, nf, tol2, nullptr, st));
        if ((it + 1) % 4 == 0 || it + 1 == maxit) {
            int h = 0;
            PAT_CUDA(cudaMemcpyAsync(&h, p->nactive, sizeof(int), cudaMemcpyDeviceToHost, st));
            PAT_CUDA(cudaStreamSynchronize(st));
            if (h == 0) {
                ++it;
                break;
            }
        }
        RC(conv(p, p->r, p->s, nf, true, st));
        RC(dot(p, p->r, p->s, nf, p->part, st));
        RC(scalar(p, 3, nf, 0.0, nullptr, st));
        k_pr_dir<<<vec_blocks(tot), 256, 0, st>>>(p->d, p->s, p->sc + SC_BETA * p->maxf, nn, nf);
        RC(chk("k_pr_dir"));
    }
    if (iters) *iters = it;
    return PAT_OK;
}

int check_fields(const pat_prior_s* p, int nf, const char* who) {
    if (!p) { set_error("%s: null prior", who); return PAT_EINVAL; }
    if (nf < 1 || nf > p->maxf) { set_error("%s: nf = %d outside 1..%d", who, nf, p->maxf); return PAT_EINVAL; }
    return PAT_OK;
}

}  // namespace

extern "C" int pat_prior_create(int n, double dx, double tau, int max_fields, pat_prior* out) {
    if (!out) { set_error("pat_prior_create: null output"); return PAT_EINVAL; }
    *out = nullptr;
    if (n < 2 || n > 512 || !(dx > 0) || !(tau > 0) || max_fields < 1 || max_fields > 1024) {
        set_error("pat_prior_create: need 2 <= n <= 512, dx > 0, tau > 0, 1 <= max_fields <= 1024");
        return PAT_EINVAL;
    }
    // Spectrum of the periodic kernel on a torus of side M: lambda = C k C (k even,
    // C_uv = cos(2 pi u v / M)), FP64.  Any M >= 2n - 1 gives Xi exactly; M grows (5-smooth
    // sizes, up to 1024) until lambda > 0, so that the preconditioner is positive definite.
    const double PI = 3.14159265358979323846;
    int M = 2 * n - 2;
    FftDesc fd{};
    std::vector<double> lam;
    double lmax = 0.0, lmin = 0.0;
    do {
        ++M;
        while (!radix_schedule(M, &fd)) ++M;
        std::vector<double> k(size_t(M) * M), cs(size_t(M) * M), t(size_t(M) * M, 0.0);
        lam.assign(size_t(M) * M, 0.0);
        for (int i = 0; i < M; ++i) {
            const int oi = i <= M / 2 ? i : i - M;
            for (int j = 0; j < M; ++j) {
                const int oj = j <= M / 2 ? j : j - M;
                k[size_t(i) * M + j] = std::exp(-dx * std::sqrt(double(oi) * oi + double(oj) * oj) / tau);
            }
        }
        for (int u = 0; u < M; ++u)
            for (int v = 0; v < M; ++v)
                cs[size_t(u) * M + v] = std::cos(2.0 * PI * double((size_t(u) * v) % M) / M);
        for (int u = 0; u < M; ++u)           // t = C k
            for (int i = 0; i < M; ++i) {
                const double c = cs[size_t(u) * M + i];
                const double* kr = &k[size_t(i) * M];
                double* tr = &t[size_t(u) * M];
                for (int j = 0; j < M; ++j) tr[j] += c * kr[j];
            }
        for (int u = 0; u < M; ++u)           // lam = t C
            for (int j = 0; j < M; ++j) {
                const double tv = t[size_t(u) * M + j];
                const double* cr = &cs[size_t(j) * M];
                double* lr = &lam[size_t(u) * M];
                for (int v = 0; v < M; ++v) lr[v] += tv * cr[v];
            }
        lmax = *std::max_element(lam.begin(), lam.end());
        lmin = *std::min_element(lam.begin(), lam.end());
    } while (!(lmin > 0.0) && M < 1024);
    pat_prior_s* p = new (std::nothrow) pat_prior_s();
    if (!p) { set_error("pat_prior_create: out of host memory"); return PAT_ENOMEM; }
    p->n = n;
    p->M = M;
    p->maxf = max_fields;
    p->dx = dx;
    p->tau = tau;
    p->fd = fd;
    cudaGetDevice(&p->device);
    p->rows_per_cta = 4;
    p->cols_per_cta = 8;
    p->smem_rows = size_t(M + 2 * p->rows_per_cta * M) * sizeof(float2);
    p->smem_cols = size_t(M + 2 * p->cols_per_cta * (M + 1)) * sizeof(float2);
    std::vector<float> hl(size_t(M) * M), hi(size_t(M) * M);
    for (size_t i = 0; i < hl.size(); ++i) {
        hl[i] = float(lam[i]);
        hi[i] = float(1.0 / std::max(lam[i], 1e-9 * lmax));   // positive definite even if M stopped at 1024
    }
    std::vector<float2> htw(M);
    for (int q = 0; q < M; ++q) htw[q] = make_float2(float(std::cos(-2.0 * PI * q / M)), float(std::sin(-2.0 * PI * q / M)));
    const size_t nn = size_t(n) * n, vecb = size_t(max_fields) * nn * sizeof(float);
    const size_t np = (size_t(max_fields) + 1) / 2;
    cudaError_t e = cudaSuccess;
    auto al = [&](void** ptr, size_t bytes) {
        if (e == cudaSuccess) e = cudaMalloc(ptr, bytes);
    };
    al((void**)&p->tw, M * sizeof(float2));
    al((void**)&p->lam, size_t(M) * M * sizeof(float));
    al((void**)&p->ilam, size_t(M) * M * sizeof(float));
    al((void**)&p->W, np * M * M * sizeof(float2));
    al((void**)&p->b, vecb);
    al((void**)&p->r, vecb);
    al((void**)&p->s, vecb);
    al((void**)&p->d, vecb);
    al((void**)&p->q, vecb);
    al((void**)&p->part, 2 * size_t(max_fields) * kDotBlocks * sizeof(double));
    al((void**)&p->sc, size_t(kSc) * max_fields * sizeof(double));
    al((void**)&p->active, max_fields * sizeof(int));
    al((void**)&p->nactive, sizeof(int));
    if (e == cudaSuccess) e = cudaMemcpy(p->tw, htw.data(), M * sizeof(float2), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(p->lam, hl.data(), hl.size() * sizeof(float), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(p->ilam, hi.data(), hi.size() * sizeof(float), cudaMemcpyHostToDevice);
    // copies from pageable memory may still be in flight when cudaMemcpy returns, and the
    // caller's non-blocking streams are not ordered after the legacy stream: wait for them
    if (e == cudaSuccess) e = cudaStreamSynchronize(cudaStreamLegacy);
    const void* kerns[] = {(const void*)k_pr_rows_fwd, (const void*)k_pr_rows_inv};
    for (const void* f : kerns)
        if (e == cudaSuccess) e = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, int(p->smem_rows));
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute((const void*)k_pr_cols, cudaFuncAttributeMaxDynamicSharedMemorySize, int(p->smem_cols));
    if (e != cudaSuccess) {
        pat_prior_destroy(p);
        return cuda_fail(e, "pat_prior_create");
    }
    *out = p;
    return PAT_OK;
}

extern "C" int pat_prior_destroy(pat_prior p) {
    if (!p) return PAT_OK;
    void* ptrs[] = {p->tw, p->lam, p->ilam, p->W, p->b, p->r, p->s, p->d, p->q, p->part, p->sc, p->active, p->nactive};
    for (void* q : ptrs)
        if (q) cudaFree(q);
    delete p;
    return PAT_OK;
}

extern "C" int pat_prior_xi(pat_prior p, const float* d_v, float* d_out, int nf, void* stream) {
    RC(check_fields(p, nf, "pat_prior_xi"));
    if (!d_v || !d_out) { set_error("pat_prior_xi: null argument"); return PAT_EINVAL; }
    return conv(p, d_v, d_out, nf, false, static_cast<cudaStream_t>(stream));
}

extern "C" int pat_prior_solve(pat_prior p, const float* d_b, float* d_z, int nf, double tol, int maxit, int warm,
                               int* h_iters, void* stream) {
    RC(check_fields(p, nf, "pat_prior_solve"));
    if (!d_b || !d_z || !(tol > 0) || maxit < 1) { set_error("pat_prior_solve: bad argument"); return PAT_EINVAL; }
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    PAT_CUDA(cudaMemcpyAsync(p->b, d_b, size_t(nf) * p->n * p->n * sizeof(float), cudaMemcpyDeviceToDevice, st));
    return pcg(p, d_z, nf, tol, maxit, warm != 0, h_iters, st);
}

extern "C" int pat_prior_eval(pat_prior p, const float* d_x, int nf, const double* h_eta, const double* h_sigma,
                              const double* h_gscale, float* d_z, float* d_grad, double* d_J, double tol, int maxit,
                              int warm, int* h_iters, void* stream) {
    RC(check_fields(p, nf, "pat_prior_eval"));
    if (!d_x || !h_eta || !h_sigma || !d_z || !(tol > 0) || maxit < 1) {
        set_error("pat_prior_eval: bad argument");
        return PAT_EINVAL;
    }
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    std::vector<double> hp(size_t(kSc) * p->maxf, 0.0);
    for (int f = 0; f < nf; ++f) {
        if (!(h_sigma[f] > 0)) { set_error("pat_prior_eval: sigma must be > 0"); return PAT_EINVAL; }
        hp[size_t(SC_ETA) * p->maxf + f] = h_eta[f];
        hp[size_t(SC_ISIG2) * p->maxf + f] = 1.0 / (h_sigma[f] * h_sigma[f]);
        hp[size_t(SC_COEF) * p->maxf + f] = (h_gscale ? h_gscale[f] : 1.0) / (h_sigma[f] * h_sigma[f]);
    }
    // eta, coefficients and 1/sigma^2 into the scalar block (rows SC_ETA .. SC_ISIG2)
    PAT_CUDA(cudaMemcpyAsync(p->sc + size_t(SC_ETA) * p->maxf, hp.data() + size_t(SC_ETA) * p->maxf,
                             3 * size_t(p->maxf) * sizeof(double), cudaMemcpyHostToDevice, st));
    const size_t nn = size_t(p->n) * p->n, tot = nn * nf;
    k_pr_axpy<<<vec_blocks(tot), 256, 0, st>>>(p->b, d_x, nullptr, p->sc + SC_ETA * p->maxf, 0.f, nn, nf);
    RC(chk("k_pr_axpy"));
    RC(pcg(p, d_z, nf, tol, maxit, warm != 0, h_iters, st));
    if (d_J) {
        RC(dot(p, p->b, d_z, nf, p->part, st));
        RC(scalar(p, 4, nf, 0.0, d_J, st));
    }
    if (d_grad) {
        k_pr_grad<<<vec_blocks(tot), 256, 0, st>>>(d_grad, d_z, p->sc + SC_COEF * p->maxf, nn, nf);
        RC(chk("k_pr_grad"));
    }
    // the host scalars must outlive the asynchronous copy
    PAT_CUDA(cudaStreamSynchronize(st));
    return PAT_OK;
}

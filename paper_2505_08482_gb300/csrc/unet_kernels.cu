// Kernels of the learned warm start (a small U-Net on BF16 tensor cores):
// a BF16 GEMM with FP32 accumulation on the warp-level tensor-core
// instructions (mma.sync m16n8k16, operands staged with cp.async and read
// with ldmatrix), im2col for 3x3 convolutions in NHWC layout, transposes,
// pooling, upsampling, concatenation, bias/ReLU, the MSE loss and Adam.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>

#include "pat_internal.h"
#include "unet.h"

namespace pat {

// ---------------------------------------------------------------------------
// GEMM  C[M][N] = A[M][K] . B[N][K]^T  (both operands K-contiguous, K % 8 == 0)
// epilogue: (+ bias[n]) (ReLU) -> bf16 or fp32 store, or fp32 atomic add (split K)
namespace gemm {
constexpr int BM = 128, BN = 128, BK = 32, STAGES = 3, PITCH = BK + 8;   // bf16 elements per smem row
constexpr int THREADS = 256;

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void cp_async16(void* smem, const void* gmem, bool valid) {
    const int sz = valid ? 16 : 0;   // zero-fill outside the matrix
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(smem_u32(smem)), "l"(gmem), "r"(sz));
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N)); }

__device__ __forceinline__ void ldmatrix_x4(uint32_t (&r)[4], const void* p) {
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];\n"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
                 : "r"(smem_u32(p)));
}
__device__ __forceinline__ void mma_bf16(float (&d)[4], const uint32_t (&a)[4], uint32_t b0, uint32_t b1) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};\n"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

struct Args {
    const __nv_bfloat16* A;
    const __nv_bfloat16* B;
    int M, N, K;
    int lda, ldb;          // row pitches (elements) of A and B
    const float* bias;     // [N] or null
    int relu;
    void* C;
    int ldc;
    int out_mode;          // 0 bf16 store, 1 fp32 store, 2 fp32 atomic add
    int ksplit;            // K range per blockIdx.z
};

__global__ void __launch_bounds__(THREADS) k_gemm(Args a) {
    extern __shared__ __align__(16) unsigned char smraw[];
    __nv_bfloat16* sA = reinterpret_cast<__nv_bfloat16*>(smraw);
    __nv_bfloat16* sB = sA + STAGES * BM * PITCH;
    const int tid = threadIdx.x, warp = tid / 32, lane = tid % 32;
    const int wm = warp / 4, wn = warp % 4;          // 2 x 4 warps, warp tile 64 x 32
    const int m0 = blockIdx.y * BM, n0 = blockIdx.x * BN;
    const int kb = blockIdx.z * a.ksplit;
    const int ke = min(a.K, kb + a.ksplit);
    const int nk = (ke - kb + BK - 1) / BK;
    float acc[4][4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j)
#pragma unroll
            for (int q = 0; q < 4; ++q) acc[i][j][q] = 0.f;

    auto load_stage = [&](int stage, int kt) {
        const int k0 = kb + kt * BK;
#pragma unroll
        for (int it = 0; it < 2; ++it) {
            const int c = tid + it * THREADS;       // 512 chunks of 8 bf16 per operand tile
            const int row = c / 4, kc = (c % 4) * 8;
            const int gk = k0 + kc;
            const bool kin = gk < ke;
            const int gm = m0 + row, gn = n0 + row;
            const bool va = kin && gm < a.M, vb = kin && gn < a.N;
            cp_async16(sA + (stage * BM + row) * PITCH + kc, a.A + (va ? size_t(gm) * a.lda + gk : 0), va);
            cp_async16(sB + (stage * BN + row) * PITCH + kc, a.B + (vb ? size_t(gn) * a.ldb + gk : 0), vb);
        }
    };
#pragma unroll
    for (int s = 0; s < STAGES - 1; ++s) {
        if (s < nk) load_stage(s, s);
        cp_async_commit();
    }
    for (int kt = 0; kt < nk; ++kt) {
        cp_async_wait<STAGES - 2>();
        __syncthreads();
        const int nxt = kt + STAGES - 1;
        if (nxt < nk) load_stage(nxt % STAGES, nxt);
        cp_async_commit();
        const __nv_bfloat16* tA = sA + (kt % STAGES) * BM * PITCH;
        const __nv_bfloat16* tB = sB + (kt % STAGES) * BN * PITCH;
#pragma unroll
        for (int kk = 0; kk < BK; kk += 16) {
            uint32_t af[4][4], bf[2][4];
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                const int row = wm * 64 + i * 16 + (lane % 16);
                ldmatrix_x4(af[i], tA + row * PITCH + kk + (lane / 16) * 8);
            }
#pragma unroll
            for (int j = 0; j < 2; ++j) {
                const int row = wn * 32 + j * 16 + (lane % 8) + (lane / 16) * 8;
                ldmatrix_x4(bf[j], tB + row * PITCH + kk + ((lane / 8) % 2) * 8);
            }
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) mma_bf16(acc[i][j], af[i], bf[j / 2][(j % 2) * 2], bf[j / 2][(j % 2) * 2 + 1]);
        }
    }
    cp_async_wait<0>();
    // epilogue
    const int g = lane / 4, t4 = lane % 4;
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j)
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int m = m0 + wm * 64 + i * 16 + g + h * 8;
                const int n = n0 + wn * 32 + j * 8 + t4 * 2;
                if (m >= a.M) continue;
#pragma unroll
                for (int e = 0; e < 2; ++e) {
                    const int nn = n + e;
                    if (nn >= a.N) continue;
                    float v = acc[i][j][h * 2 + e];
                    if (a.bias) v += a.bias[nn];
                    if (a.relu) v = fmaxf(v, 0.f);
                    const size_t o = size_t(m) * a.ldc + nn;
                    if (a.out_mode == 0)
                        static_cast<__nv_bfloat16*>(a.C)[o] = __float2bfloat16(v);
                    else if (a.out_mode == 1)
                        static_cast<float*>(a.C)[o] = v;
                    else
                        atomicAdd(static_cast<float*>(a.C) + o, v);
                }
            }
}
}  // namespace gemm

int unet_gemm(cudaStream_t st, const __nv_bfloat16* A, int lda, const __nv_bfloat16* B, int ldb, int M, int N,
              int K, const float* bias, int relu, void* C, int ldc, int out_mode, int splitk) {
    if (K % 8 || lda % 8 || ldb % 8 || M <= 0 || N <= 0 || K <= 0) {
        set_error("unet_gemm: K and the operand pitches must be multiples of 8 (M=%d N=%d K=%d)", M, N, K);
        return PAT_EINVAL;
    }
    static bool configured = false;
    const size_t smem = size_t(gemm::STAGES) * (gemm::BM + gemm::BN) * gemm::PITCH * sizeof(__nv_bfloat16);
    if (!configured) {
        PAT_CUDA(cudaFuncSetAttribute(gemm::k_gemm, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem)));
        configured = true;
    }
    splitk = splitk < 1 ? 1 : splitk;
    int ks = (K + splitk - 1) / splitk;
    ks = (ks + gemm::BK - 1) / gemm::BK * gemm::BK;
    const int nz = (K + ks - 1) / ks;
    gemm::Args a{A, B, M, N, K, lda, ldb, bias, relu, C, ldc, out_mode, ks};
    dim3 grid((N + gemm::BN - 1) / gemm::BN, (M + gemm::BM - 1) / gemm::BM, nz);
    count_launch();
    gemm::k_gemm<<<grid, gemm::THREADS, smem, st>>>(a);
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? PAT_OK : cuda_fail(e, "k_gemm");
}

// ---------------------------------------------------------------------------
// elementwise / layout kernels (NHWC, channel counts padded to multiples of 8)
static unsigned nblk(size_t n) {
    size_t b = (n + 255) / 256;
    return unsigned(b > 65535 * 8 ? 65535 * 8 : (b < 1 ? 1 : b));
}
#define GRID_STRIDE(i, n) for (size_t i = size_t(blockIdx.x) * blockDim.x + threadIdx.x; i < (n); i += size_t(gridDim.x) * blockDim.x)

// col[b][y][x][tap][c] = in[b][y+dy][x+dx][c] (zero outside), tap = (dy+1)*3 + (dx+1); flip: tap -> 8 - tap
__global__ void k_im2col(const __nv_bfloat16* __restrict__ in, __nv_bfloat16* __restrict__ col, int B, int H, int W,
                         int C, int ldc_in, int flip) {
    const size_t total = size_t(B) * H * W * 9 * C;
    GRID_STRIDE(i, total) {
        const int c = int(i % C);
        size_t r = i / C;
        int tap = int(r % 9);
        r /= 9;
        const int x = int(r % W);
        r /= W;
        const int y = int(r % H);
        const int b = int(r / H);
        const int t = flip ? 8 - tap : tap;
        const int yy = y + t / 3 - 1, xx = x + t % 3 - 1;
        __nv_bfloat16 v = __float2bfloat16(0.f);
        if (yy >= 0 && yy < H && xx >= 0 && xx < W) v = in[((size_t(b) * H + yy) * W + xx) * ldc_in + c];
        col[i] = v;
    }
}

// out[c][r] = in[r][c] for an R x C bf16 matrix with row pitch ld
__global__ void k_transpose(const __nv_bfloat16* __restrict__ in, __nv_bfloat16* __restrict__ out, int R, int C,
                            int ld) {
    __shared__ __nv_bfloat16 t[32][33];
    for (int bx = blockIdx.x; bx < (C + 31) / 32; bx += gridDim.x)
        for (int by = blockIdx.y; by < (R + 31) / 32; by += gridDim.y) {
            const int c = bx * 32 + threadIdx.x;
            for (int j = threadIdx.y; j < 32; j += blockDim.y) {
                const int r = by * 32 + j;
                t[j][threadIdx.x] = (r < R && c < C) ? in[size_t(r) * ld + c] : __float2bfloat16(0.f);
            }
            __syncthreads();
            const int r2 = by * 32 + threadIdx.x;
            for (int j = threadIdx.y; j < 32; j += blockDim.y) {
                const int c2 = bx * 32 + j;
                if (c2 < C && r2 < R) out[size_t(c2) * R + r2] = t[threadIdx.x][j];
            }
            __syncthreads();
        }
}

// 2x2 max pooling (NHWC); idx records the argmax (0..3) for the backward
__global__ void k_maxpool(const __nv_bfloat16* __restrict__ in, __nv_bfloat16* __restrict__ out,
                          unsigned char* __restrict__ idx, int B, int H, int W, int C) {
    const int Ho = H / 2, Wo = W / 2;
    const size_t total = size_t(B) * Ho * Wo * C;
    GRID_STRIDE(i, total) {
        const int c = int(i % C);
        size_t r = i / C;
        const int x = int(r % Wo);
        r /= Wo;
        const int y = int(r % Ho);
        const int b = int(r / Ho);
        float best = -3.0e38f;
        int bi = 0;
        for (int q = 0; q < 4; ++q) {
            const float v = __bfloat162float(in[((size_t(b) * H + 2 * y + q / 2) * W + 2 * x + q % 2) * C + c]);
            if (v > best) {
                best = v;
                bi = q;
            }
        }
        out[i] = __float2bfloat16(best);
        idx[i] = (unsigned char)bi;
    }
}

__global__ void k_maxpool_bwd(const __nv_bfloat16* __restrict__ dout, const unsigned char* __restrict__ idx,
                              __nv_bfloat16* __restrict__ din, int B, int H, int W, int C) {
    const int Ho = H / 2, Wo = W / 2;
    const size_t total = size_t(B) * Ho * Wo * C;
    GRID_STRIDE(i, total) {
        const int c = int(i % C);
        size_t r = i / C;
        const int x = int(r % Wo);
        r /= Wo;
        const int y = int(r % Ho);
        const int b = int(r / Ho);
        for (int q = 0; q < 4; ++q)
            din[((size_t(b) * H + 2 * y + q / 2) * W + 2 * x + q % 2) * C + c] =
                q == idx[i] ? dout[i] : __float2bfloat16(0.f);
    }
}

// nearest 2x upsampling of src (C channels, pitch ldi) into dst channels [off, off+C) of pitch ldo
__global__ void k_upsample(const __nv_bfloat16* __restrict__ src, __nv_bfloat16* __restrict__ dst, int B, int Hs,
                           int Ws, int C, int ldi, int ldo, int off) {
    const int H = Hs * 2, W = Ws * 2;
    const size_t total = size_t(B) * H * W * C;
    GRID_STRIDE(i, total) {
        const int c = int(i % C);
        size_t r = i / C;
        const int x = int(r % W);
        r /= W;
        const int y = int(r % H);
        const int b = int(r / H);
        dst[((size_t(b) * H + y) * W + x) * ldo + off + c] = src[((size_t(b) * Hs + y / 2) * Ws + x / 2) * ldi + c];
    }
}

// backward of the nearest upsampling: sum of the 4 children (fp32 math)
__global__ void k_upsample_bwd(const __nv_bfloat16* __restrict__ dst, __nv_bfloat16* __restrict__ dsrc, int B,
                               int Hs, int Ws, int C, int ldo, int off) {
    const int H = Hs * 2, W = Ws * 2;
    const size_t total = size_t(B) * Hs * Ws * C;
    GRID_STRIDE(i, total) {
        const int c = int(i % C);
        size_t r = i / C;
        const int x = int(r % Ws);
        r /= Ws;
        const int y = int(r % Hs);
        const int b = int(r / Hs);
        float s = 0.f;
        for (int q = 0; q < 4; ++q)
            s += __bfloat162float(dst[((size_t(b) * H + 2 * y + q / 2) * W + 2 * x + q % 2) * ldo + off + c]);
        dsrc[i] = __float2bfloat16(s);
    }
}

// copy channels: dst[p][off + c] = src[p][c] (c < C), pitches lds / ldd; back: src <- dst slice
__global__ void k_copy_ch(const __nv_bfloat16* __restrict__ src, __nv_bfloat16* __restrict__ dst, size_t P, int C,
                          int lds, int ldd, int off) {
    GRID_STRIDE(i, P * C) {
        const size_t p = i / C;
        const int c = int(i % C);
        dst[p * ldd + off + c] = src[p * lds + c];
    }
}

// dst[p][c] += src[p][off + c]
__global__ void k_add_ch(__nv_bfloat16* __restrict__ dst, const __nv_bfloat16* __restrict__ src, size_t P, int C,
                         int lds, int off) {
    GRID_STRIDE(i, P * C) {
        const size_t p = i / C;
        const int c = int(i % C);
        dst[i] = __float2bfloat16(__bfloat162float(dst[i]) + __bfloat162float(src[p * lds + off + c]));
    }
}

// weights for the data gradient: Wt[ci][tap][co] = W[co][tap][ci]
__global__ void k_weight_t(const __nv_bfloat16* __restrict__ W, __nv_bfloat16* __restrict__ Wt, int Cout, int Cin) {
    const size_t total = size_t(Cout) * 9 * Cin;
    GRID_STRIDE(i, total) {
        const int ci = int(i % Cin);
        size_t r = i / Cin;
        const int tap = int(r % 9);
        const int co = int(r / 9);
        Wt[(size_t(ci) * 9 + tap) * Cout + co] = W[i];
    }
}

// ReLU backward in place: g *= (y > 0)
__global__ void k_relu_bwd(__nv_bfloat16* __restrict__ g, const __nv_bfloat16* __restrict__ y, size_t n) {
    GRID_STRIDE(i, n) {
        if (!(__bfloat162float(y[i]) > 0.f)) g[i] = __float2bfloat16(0.f);
    }
}

// bias gradient: db[c] = sum_p g[p][c] (row pitch ld; one block per channel, fixed order)
__global__ void k_bias_grad(const __nv_bfloat16* __restrict__ g, float* __restrict__ db, size_t P, int C, int ld) {
    __shared__ float red[256];
    for (int c = blockIdx.x; c < C; c += gridDim.x) {
        float s = 0.f;
        for (size_t p = threadIdx.x; p < P; p += blockDim.x) s += __bfloat162float(g[p * ld + c]);
        red[threadIdx.x] = s;
        __syncthreads();
        for (int w = 128; w > 0; w >>= 1) {
            if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
            __syncthreads();
        }
        if (threadIdx.x == 0) db[c] = red[0];
        __syncthreads();
    }
}

// MSE loss L = mean (pred - target)^2 over n values; grad[i * ld] = 2 (pred - target) / n (bf16)
__global__ void k_mse(const float* __restrict__ pred, const float* __restrict__ tgt, __nv_bfloat16* __restrict__ grad,
                      size_t n, int ld, double* __restrict__ loss_part) {
    __shared__ double red[256];
    double s = 0.0;
    for (size_t i = size_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += size_t(gridDim.x) * blockDim.x) {
        const float d = pred[i] - tgt[i];
        s += double(d) * d;
        grad[i * ld] = __float2bfloat16(2.f * d / float(n));
    }
    red[threadIdx.x] = s;
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
        if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) loss_part[blockIdx.x] = red[0];
}

__global__ void k_sum_d(const double* __restrict__ part, int n, double* __restrict__ out, double scale) {
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        double s = 0.0;
        for (int i = 0; i < n; ++i) s += part[i];
        *out = s * scale;
    }
}

// Adam on fp32 master weights, refreshing the bf16 copies
__global__ void k_adam(float* __restrict__ w, __nv_bfloat16* __restrict__ wb, const float* __restrict__ g,
                       float* __restrict__ m, float* __restrict__ v, size_t n, float lr, float b1, float b2, float eps,
                       float bc1, float bc2) {
    GRID_STRIDE(i, n) {
        const float gi = g[i];
        const float mi = b1 * m[i] + (1.f - b1) * gi;
        const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
        m[i] = mi;
        v[i] = vi;
        const float wi = w[i] - lr * (mi / bc1) / (sqrtf(vi / bc2) + eps);
        w[i] = wi;
        if (wb) wb[i] = __float2bfloat16(wi);
    }
}

__global__ void k_f32_to_bf16(const float* __restrict__ a, __nv_bfloat16* __restrict__ b, size_t n) {
    GRID_STRIDE(i, n) b[i] = __float2bfloat16(a[i]);
}

__global__ void k_bf16_to_f32(const __nv_bfloat16* __restrict__ a, float* __restrict__ b, size_t n, int lda) {
    GRID_STRIDE(i, n) b[i] = __bfloat162float(a[i * lda]);
}

// input staging: fp32 [B][Cin][H][W] (NCHW, as the solver produces images) -> bf16 NHWC with C padded
__global__ void k_pack_input(const float* __restrict__ in, __nv_bfloat16* __restrict__ out, int B, int Cin, int H,
                             int W, int Cp) {
    const size_t total = size_t(B) * H * W * Cp;
    GRID_STRIDE(i, total) {
        const int c = int(i % Cp);
        size_t r = i / Cp;
        const int x = int(r % W);
        r /= W;
        const int y = int(r % H);
        const int b = int(r / H);
        out[i] = c < Cin ? __float2bfloat16(in[((size_t(b) * Cin + c) * H + y) * W + x]) : __float2bfloat16(0.f);
    }
}

// ---- launchers ----
#define LAUNCH_CHECK(name)                                                        \
    do {                                                                          \
        count_launch();                                                           \
        cudaError_t e_ = cudaGetLastError();                                      \
        if (e_ != cudaSuccess) return cuda_fail(e_, name);                        \
    } while (0)

int unet_im2col(cudaStream_t st, const __nv_bfloat16* in, __nv_bfloat16* col, int B, int H, int W, int C, int ldc_in,
                int flip) {
    k_im2col<<<nblk(size_t(B) * H * W * 9 * C), 256, 0, st>>>(in, col, B, H, W, C, ldc_in, flip);
    LAUNCH_CHECK("k_im2col");
    return PAT_OK;
}
int unet_transpose(cudaStream_t st, const __nv_bfloat16* in, __nv_bfloat16* out, int R, int C, int ld) {
    dim3 grid(std::min((C + 31) / 32, 1024), std::min((R + 31) / 32, 1024));
    k_transpose<<<grid, dim3(32, 8), 0, st>>>(in, out, R, C, ld);
    LAUNCH_CHECK("k_transpose");
    return PAT_OK;
}
int unet_maxpool(cudaStream_t st, const __nv_bfloat16* in, __nv_bfloat16* out, unsigned char* idx, int B, int H, int W,
                 int C) {
    k_maxpool<<<nblk(size_t(B) * H * W * C / 4), 256, 0, st>>>(in, out, idx, B, H, W, C);
    LAUNCH_CHECK("k_maxpool");
    return PAT_OK;
}
int unet_maxpool_bwd(cudaStream_t st, const __nv_bfloat16* dout, const unsigned char* idx, __nv_bfloat16* din, int B,
                     int H, int W, int C) {
    k_maxpool_bwd<<<nblk(size_t(B) * H * W * C / 4), 256, 0, st>>>(dout, idx, din, B, H, W, C);
    LAUNCH_CHECK("k_maxpool_bwd");
    return PAT_OK;
}
int unet_upsample(cudaStream_t st, const __nv_bfloat16* src, __nv_bfloat16* dst, int B, int Hs, int Ws, int C, int ldi,
                  int ldo, int off) {
    k_upsample<<<nblk(size_t(B) * Hs * Ws * 4 * C), 256, 0, st>>>(src, dst, B, Hs, Ws, C, ldi, ldo, off);
    LAUNCH_CHECK("k_upsample");
    return PAT_OK;
}
int unet_upsample_bwd(cudaStream_t st, const __nv_bfloat16* dst, __nv_bfloat16* dsrc, int B, int Hs, int Ws, int C,
                      int ldo, int off) {
    k_upsample_bwd<<<nblk(size_t(B) * Hs * Ws * C), 256, 0, st>>>(dst, dsrc, B, Hs, Ws, C, ldo, off);
    LAUNCH_CHECK("k_upsample_bwd");
    return PAT_OK;
}
int unet_copy_ch(cudaStream_t st, const __nv_bfloat16* src, __nv_bfloat16* dst, size_t P, int C, int lds, int ldd,
                 int off) {
    k_copy_ch<<<nblk(P * C), 256, 0, st>>>(src, dst, P, C, lds, ldd, off);
    LAUNCH_CHECK("k_copy_ch");
    return PAT_OK;
}
int unet_add_ch(cudaStream_t st, __nv_bfloat16* dst, const __nv_bfloat16* src, size_t P, int C, int lds, int off) {
    k_add_ch<<<nblk(P * C), 256, 0, st>>>(dst, src, P, C, lds, off);
    LAUNCH_CHECK("k_add_ch");
    return PAT_OK;
}
int unet_weight_t(cudaStream_t st, const __nv_bfloat16* W, __nv_bfloat16* Wt, int Cout, int Cin) {
    k_weight_t<<<nblk(size_t(Cout) * 9 * Cin), 256, 0, st>>>(W, Wt, Cout, Cin);
    LAUNCH_CHECK("k_weight_t");
    return PAT_OK;
}
int unet_relu_bwd(cudaStream_t st, __nv_bfloat16* g, const __nv_bfloat16* y, size_t n) {
    k_relu_bwd<<<nblk(n), 256, 0, st>>>(g, y, n);
    LAUNCH_CHECK("k_relu_bwd");
    return PAT_OK;
}
int unet_bias_grad(cudaStream_t st, const __nv_bfloat16* g, float* db, size_t P, int C, int ld) {
    k_bias_grad<<<std::min(C, 1024), 256, 0, st>>>(g, db, P, C, ld);
    LAUNCH_CHECK("k_bias_grad");
    return PAT_OK;
}
int unet_mse(cudaStream_t st, const float* pred, const float* tgt, __nv_bfloat16* grad, size_t n, int ld,
             double* part, double* loss) {
    k_mse<<<256, 256, 0, st>>>(pred, tgt, grad, n, ld, part);
    LAUNCH_CHECK("k_mse");
    k_sum_d<<<1, 32, 0, st>>>(part, 256, loss, 1.0 / double(n));
    LAUNCH_CHECK("k_sum_d");
    return PAT_OK;
}
int unet_adam(cudaStream_t st, float* w, __nv_bfloat16* wb, const float* g, float* m, float* v, size_t n, float lr,
              float b1, float b2, float eps, float bc1, float bc2) {
    k_adam<<<nblk(n), 256, 0, st>>>(w, wb, g, m, v, n, lr, b1, b2, eps, bc1, bc2);
    LAUNCH_CHECK("k_adam");
    return PAT_OK;
}
int unet_f32_to_bf16(cudaStream_t st, const float* a, __nv_bfloat16* b, size_t n) {
    k_f32_to_bf16<<<nblk(n), 256, 0, st>>>(a, b, n);
    LAUNCH_CHECK("k_f32_to_bf16");
    return PAT_OK;
}
int unet_bf16_to_f32(cudaStream_t st, const __nv_bfloat16* a, float* b, size_t n, int lda) {
    k_bf16_to_f32<<<nblk(n), 256, 0, st>>>(a, b, n, lda);
    LAUNCH_CHECK("k_bf16_to_f32");
    return PAT_OK;
}
int unet_pack_input(cudaStream_t st, const float* in, __nv_bfloat16* out, int B, int Cin, int H, int W, int Cp) {
    k_pack_input<<<nblk(size_t(B) * H * W * Cp), 256, 0, st>>>(in, out, B, Cin, H, W, Cp);
    LAUNCH_CHECK("k_pack_input");
    return PAT_OK;
}

}  // namespace pat

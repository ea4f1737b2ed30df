// Kernel launchers of the learned warm start (unet_kernels.cu).
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cstddef>

namespace pat {

// C[M][N] = A[M][K] . B[N][K]^T (+bias)(ReLU); out_mode 0 bf16, 1 fp32, 2 fp32 atomic add (split K)
int unet_gemm(cudaStream_t st, const __nv_bfloat16* A, int lda, const __nv_bfloat16* B, int ldb, int M, int N,
              int K, const float* bias, int relu, void* C, int ldc, int out_mode, int splitk);
// the same GEMM on tcgen05 / TMEM / TMA (unet_tc05.cu); supported: K >= 64, pitches multiples of 8,
// 16-byte aligned operands.  d_status (may be null) gets PAT_STATUS_TC05 if a bounded wait gave up.
bool unet_gemm_tc05_supported(const __nv_bfloat16* A, int lda, const __nv_bfloat16* B, int ldb, int M, int N, int K);
int unet_gemm_tc05(cudaStream_t st, const __nv_bfloat16* A, int lda, const __nv_bfloat16* B, int ldb, int M, int N,
                   int K, const float* bias, int relu, void* C, int ldc, int out_mode, int splitk, int* d_status);
int unet_im2col(cudaStream_t st, const __nv_bfloat16* in, __nv_bfloat16* col, int B, int H, int W, int C, int ldc_in,
                int flip);
int unet_transpose(cudaStream_t st, const __nv_bfloat16* in, __nv_bfloat16* out, int R, int C, int ld);
int unet_maxpool(cudaStream_t st, const __nv_bfloat16* in, __nv_bfloat16* out, unsigned char* idx, int B, int H, int W,
                 int C);
int unet_maxpool_bwd(cudaStream_t st, const __nv_bfloat16* dout, const unsigned char* idx, __nv_bfloat16* din, int B,
                     int H, int W, int C);
int unet_upsample(cudaStream_t st, const __nv_bfloat16* src, __nv_bfloat16* dst, int B, int Hs, int Ws, int C, int ldi,
                  int ldo, int off);
int unet_upsample_bwd(cudaStream_t st, const __nv_bfloat16* dst, __nv_bfloat16* dsrc, int B, int Hs, int Ws, int C,
                      int ldo, int off);
int unet_copy_ch(cudaStream_t st, const __nv_bfloat16* src, __nv_bfloat16* dst, size_t P, int C, int lds, int ldd,
                 int off);
int unet_add_ch(cudaStream_t st, __nv_bfloat16* dst, const __nv_bfloat16* src, size_t P, int C, int lds, int off);
int unet_relu_bwd(cudaStream_t st, __nv_bfloat16* g, const __nv_bfloat16* y, size_t n);
int unet_bias_grad(cudaStream_t st, const __nv_bfloat16* g, float* db, size_t P, int C, int ld);
int unet_mse(cudaStream_t st, const float* pred, const float* tgt, __nv_bfloat16* grad, size_t n, int ld,
             double* part, double* loss);
int unet_adam(cudaStream_t st, float* w, __nv_bfloat16* wb, const float* g, float* m, float* v, size_t n, float lr,
              float b1, float b2, float eps, float bc1, float bc2);
int unet_f32_to_bf16(cudaStream_t st, const float* a, __nv_bfloat16* b, size_t n);
int unet_bf16_to_f32(cudaStream_t st, const __nv_bfloat16* a, float* b, size_t n, int lda);
int unet_pack_input(cudaStream_t st, const float* in, __nv_bfloat16* out, int B, int Cin, int H, int W, int Cp);
int unet_weight_t(cudaStream_t st, const __nv_bfloat16* W, __nv_bfloat16* Wt, int Cout, int Cin);

}  // namespace pat

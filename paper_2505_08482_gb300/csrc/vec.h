// Vector kernels of the optimiser and the multigrid schedule (see vec.cu).
#pragma once

#include <cuda_runtime.h>

#include <cstddef>

namespace pat {

// Box bounds and block scales of the two blocks (p0 block: indices < n0, c block: the rest),
// in block-scaled units.
struct Box {
    float lo0, hi0, s0;
    float lo1, hi1, s1;
};

int vdot(cudaStream_t st, const float* a, const float* b, size_t n, double* out, double* part,
         const double* scale = nullptr, double mul = 1.0);
int vaxpy_dev(cudaStream_t st, float* y, const float* x, size_t n, const double* coef, const double* coef2,
              float sign);
int vscale_dev(cudaStream_t st, float* y, const float* x, size_t n, const double* coef, float sign);
int vaxpby(cudaStream_t st, float* out, float a, const float* x, float b, const float* y, size_t n);
int vfill(cudaStream_t st, float* y, float v, size_t n);
int vblockscale(cudaStream_t st, float* out, const float* v, size_t n, size_t n0, float s0, float s1, int divide);
int vproject(cudaStream_t st, float* zt, float* xt, const float* z, const float* d, float alpha, size_t n,
             size_t n0, const Box& box);
int vclip_dir(cudaStream_t st, float* d, const float* z, size_t n, size_t n0, const Box& box);
int vabsmax(cudaStream_t st, const float* a, size_t n, double* out, double* part);
int vresample(cudaStream_t st, const float* src, float* dst, int nb, int ns, int nd);
int vtime_interp(cudaStream_t st, const float* y, float* out, int K, int nts, int ntd, int m, double dts,
                 double dtd);

}  // namespace pat

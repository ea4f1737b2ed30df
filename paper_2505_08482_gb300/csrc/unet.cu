// The learned warm start: a U-Net mapping the K back-projected images
// (adjoint solves at a constant speed of sound) to an initial speed of sound
// map, trained on pairs that the forward and adjoint solvers generate.
//
// Architecture (levels L, base width F): encoder level l has two 3x3
// convolutions with ReLU and F 2^l channels, followed by 2x2 max pooling
// (none after the deepest level); decoder level l upsamples the level below
// (nearest, 2x), concatenates the encoder output of level l, and applies two
// 3x3 convolutions with ReLU and F 2^l channels; a 1x1 convolution gives the
// single output channel.  Activations are BF16 NHWC with channel counts
// padded to multiples of 8; every convolution is im2col + one tensor-core
// GEMM (forward), im2col of the output gradient with flipped taps + GEMM
// (data gradient) and a split-K GEMM of transposed operands (weight
// gradient), FP32 accumulation throughout; parameters are FP32 masters with
// BF16 copies, updated by Adam.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <vector>

#include "pat_internal.h"
#include "unet.h"

using namespace pat;

namespace {

#define RC(x)                          \
    do {                               \
        int rc_ = (x);                 \
        if (rc_ != PAT_OK) return rc_; \
    } while (0)

int pad8(int c) { return (c + 7) / 8 * 8; }

struct Conv {
    int cin, cout, H, W, k;      // k = 3 or 1 (1: no im2col)
    size_t w_off, b_off;         // offsets into the fp32 parameter array
    size_t wb_off;               // offset into the bf16 weight copies
    size_t nw() const { return size_t(cout) * k * k * cin; }
};

struct Act {  // one activation buffer [B][H][W][C] (bf16) with its gradient
    int H, W, C;
    __nv_bfloat16* y = nullptr;
    __nv_bfloat16* g = nullptr;
};

}  // namespace

struct pat_unet_s {
    int levels, base, in_ch, cin_pad, H, W, maxB;
    std::vector<Conv> convs;
    size_t nparam = 0, nweight_bf = 0;
    float *param = nullptr, *grad = nullptr, *m = nullptr, *v = nullptr;
    __nv_bfloat16* wbf = nullptr;        // bf16 weights (GEMM B operands)
    __nv_bfloat16* wt = nullptr;         // scratch: transposed weights for the data gradient
    __nv_bfloat16* col = nullptr;        // scratch: im2col / transposes
    __nv_bfloat16* colt = nullptr;
    __nv_bfloat16* dt = nullptr;         // scratch: transposed output gradient
    size_t col_elems = 0;
    std::vector<Act> acts;               // activations in forward order
    std::vector<unsigned char*> pidx;    // pooling indices per encoder level
    float* out = nullptr;                // [B][H][W] fp32 prediction
    double* part = nullptr;
    double* loss = nullptr;
    long long step = 0;
    std::vector<void*> allocs;
    int device = 0;
    int gemm_path = 1;                   // 1 tcgen05 / TMEM / TMA (default), 0 warp-level tensor cores (mma.sync)
    int* status = nullptr;               // device status word of the tcgen05 GEMMs (PAT_STATUS_TC05)
};

namespace {

template <class T>
int dalloc(pat_unet_s* u, T** p, size_t n) {
    void* v = nullptr;
    cudaError_t e = cudaMalloc(&v, std::max<size_t>(n * sizeof(T), 256));
    if (e != cudaSuccess) return cuda_fail(e, "cudaMalloc(unet)");
    u->allocs.push_back(v);
    *p = static_cast<T*>(v);
    return PAT_OK;
}

// one GEMM of the network on the selected tensor-core path (tcgen05 where its operands allow)
int net_gemm(pat_unet_s* u, cudaStream_t st, const __nv_bfloat16* A, int lda, const __nv_bfloat16* B, int ldb, int M,
             int N, int K, const float* bias, int relu, void* C, int ldc, int out_mode, int splitk) {
    if (u->gemm_path == 1 && unet_gemm_tc05_supported(A, lda, B, ldb, M, N, K))
        return unet_gemm_tc05(st, A, lda, B, ldb, M, N, K, bias, relu, C, ldc, out_mode, splitk, u->status);
    return unet_gemm(st, A, lda, B, ldb, M, N, K, bias, relu, C, ldc, out_mode, splitk);
}

// conv forward: out = ReLU(conv(in) + b) (relu=0 for the final 1x1)
int conv_fwd(pat_unet_s* u, cudaStream_t st, const Conv& c, const __nv_bfloat16* in, int ldin, int B, void* out,
             int out_mode, int relu) {
    const int P = B * c.H * c.W;
    const __nv_bfloat16* wb = u->wbf + c.wb_off;
    const float* bias = u->param + c.b_off;
    if (c.k == 3) {
        RC(unet_im2col(st, in, u->col, B, c.H, c.W, c.cin, ldin, 0));
        return net_gemm(u, st, u->col, 9 * c.cin, wb, 9 * c.cin, P, c.cout, 9 * c.cin, bias, relu, out, c.cout,
                         out_mode, 1);
    }
    return net_gemm(u, st, in, ldin, wb, c.cin, P, c.cout, c.cin, bias, relu, out, c.cout, out_mode, 1);
}

// conv backward: given dz = dL/d(pre-activation) [P][cout], accumulate the parameter gradients
// and (if din) write dL/din [P][cin] (pitch ldin_out)
int conv_bwd(pat_unet_s* u, cudaStream_t st, const Conv& c, const __nv_bfloat16* in, int ldin, int B,
             const __nv_bfloat16* dz, __nv_bfloat16* din) {
    const int P = B * c.H * c.W;
    const int K1 = c.k * c.k * c.cin;
    float* dW = u->grad + c.w_off;
    float* db = u->grad + c.b_off;
    RC(unet_bias_grad(st, dz, db, size_t(P), c.cout, c.cout));
    // weight gradient: dW[co][k] = sum_p dz[p][co] col[p][k]  (transposed operands, split K over pixels)
    RC(unet_transpose(st, dz, u->dt, P, c.cout, c.cout));
    if (c.k == 3) {
        RC(unet_im2col(st, in, u->col, B, c.H, c.W, c.cin, ldin, 0));
        RC(unet_transpose(st, u->col, u->colt, P, K1, K1));
    } else {
        RC(unet_transpose(st, in, u->colt, P, K1, ldin));
    }
    PAT_CUDA(cudaMemsetAsync(dW, 0, c.nw() * sizeof(float), st));
    const int splitk = std::max(1, std::min(64, P / 4096));
    RC(net_gemm(u, st, u->dt, P, u->colt, P, c.cout, K1, P, nullptr, 0, dW, K1, 2, splitk));
    if (!din) return PAT_OK;
    // data gradient: din[p][ci] = sum_{tap,co} dz[p - off(tap)][co] W[co][tap][ci]
    if (c.k == 3) {
        RC(unet_weight_t(st, u->wbf + c.wb_off, u->wt, c.cout, c.cin));
        RC(unet_im2col(st, dz, u->col, B, c.H, c.W, c.cout, c.cout, 1));
        return net_gemm(u, st, u->col, 9 * c.cout, u->wt, 9 * c.cout, P, c.cin, 9 * c.cout, nullptr, 0, din, c.cin,
                         0, 1);
    }
    return PAT_EINVAL;
}

// activation indices: enc[l] conv a/b -> 2l, 2l+1; pooled outputs follow; see build()
struct Layout {
    std::vector<int> enc_a, enc_b, pool, dec_cat, dec_a, dec_b;
    int input = 0, final_conv = 0;
};

Layout layout_of(const pat_unet_s* u) {
    Layout L;
    int a = 0;
    L.input = a++;
    for (int l = 0; l < u->levels; ++l) {
        L.enc_a.push_back(a++);
        L.enc_b.push_back(a++);
        if (l < u->levels - 1) L.pool.push_back(a++);
    }
    for (int l = u->levels - 2; l >= 0; --l) {
        L.dec_cat.push_back(a++);
        L.dec_a.push_back(a++);
        L.dec_b.push_back(a++);
    }
    return L;
}

int forward(pat_unet_s* u, cudaStream_t st, const float* d_in, int B) {
    Layout L = layout_of(u);
    auto& A = u->acts;
    RC(unet_pack_input(st, d_in, A[L.input].y, B, u->in_ch, u->H, u->W, u->cin_pad));
    int ci = 0;
    const Act* prev = &A[L.input];
    for (int l = 0; l < u->levels; ++l) {
        RC(conv_fwd(u, st, u->convs[ci++], prev->y, prev->C, B, A[L.enc_a[l]].y, 0, 1));
        RC(conv_fwd(u, st, u->convs[ci++], A[L.enc_a[l]].y, A[L.enc_a[l]].C, B, A[L.enc_b[l]].y, 0, 1));
        prev = &A[L.enc_b[l]];
        if (l < u->levels - 1) {
            const Act& pa = A[L.pool[l]];
            RC(unet_maxpool(st, prev->y, pa.y, u->pidx[l], B, prev->H, prev->W, prev->C));
            prev = &pa;
        }
    }
    for (int d = 0; d < u->levels - 1; ++d) {
        const int l = u->levels - 2 - d;
        const Act& cat = A[L.dec_cat[d]];
        const Act& skip = A[L.enc_b[l]];
        RC(unet_upsample(st, prev->y, cat.y, B, prev->H, prev->W, prev->C, prev->C, cat.C, 0));
        RC(unet_copy_ch(st, skip.y, cat.y, size_t(B) * skip.H * skip.W, skip.C, skip.C, cat.C, prev->C));
        RC(conv_fwd(u, st, u->convs[ci++], cat.y, cat.C, B, A[L.dec_a[d]].y, 0, 1));
        RC(conv_fwd(u, st, u->convs[ci++], A[L.dec_a[d]].y, A[L.dec_a[d]].C, B, A[L.dec_b[d]].y, 0, 1));
        prev = &A[L.dec_b[d]];
    }
    return conv_fwd(u, st, u->convs[ci], prev->y, prev->C, B, u->out, 1, 0);
}

int check_batch(const pat_unet_s* u, int B) {
    if (B < 1 || B > u->maxB) {
        set_error("pat_unet: batch %d outside [1, %d]", B, u->maxB);
        return PAT_EINVAL;
    }
    return PAT_OK;
}

}  // namespace

extern "C" int pat_unet_create(pat_unet* out, int levels, int base, int in_ch, int H, int W, int max_batch) {
    if (!out) { set_error("pat_unet_create: null argument"); return PAT_EINVAL; }
    *out = nullptr;
    if (levels < 1 || levels > 6 || base < 8 || base % 8 || in_ch < 1 || max_batch < 1 || H < 8 || W < 8 ||
        H % (1 << (levels - 1)) || W % (1 << (levels - 1))) {
        set_error("pat_unet_create: need 1<=levels<=6, base a multiple of 8, H and W divisible by 2^(levels-1)");
        return PAT_EINVAL;
    }
    pat_unet_s* u = new pat_unet_s();
    u->levels = levels;
    u->base = base;
    u->in_ch = in_ch;
    u->cin_pad = pad8(in_ch);
    u->H = H;
    u->W = W;
    u->maxB = max_batch;
    cudaGetDevice(&u->device);
    // convolutions in forward order
    auto add = [&](int cin, int cout, int h, int w, int k) {
        Conv c{cin, cout, h, w, k, 0, 0, 0};
        c.w_off = u->nparam;
        u->nparam += c.nw();
        c.b_off = u->nparam;
        u->nparam += cout;
        c.wb_off = u->nweight_bf;
        u->nweight_bf += c.nw();
        u->convs.push_back(c);
    };
    int cprev = u->cin_pad;
    for (int l = 0; l < levels; ++l) {
        const int ch = base << l, h = H >> l, w = W >> l;
        add(cprev, ch, h, w, 3);
        add(ch, ch, h, w, 3);
        cprev = ch;
    }
    for (int l = levels - 2; l >= 0; --l) {
        const int ch = base << l, h = H >> l, w = W >> l;
        add(cprev + ch, ch, h, w, 3);
        add(ch, ch, h, w, 3);
        cprev = ch;
    }
    add(cprev, 1, H, W, 1);
    // activations
    auto act = [&](int h, int w, int c) {
        Act a;
        a.H = h;
        a.W = w;
        a.C = c;
        u->acts.push_back(a);
    };
    act(H, W, u->cin_pad);
    for (int l = 0; l < levels; ++l) {
        const int ch = base << l, h = H >> l, w = W >> l;
        act(h, w, ch);
        act(h, w, ch);
        if (l < levels - 1) act(h / 2, w / 2, ch);
    }
    int cb = base << (levels - 1);
    for (int l = levels - 2; l >= 0; --l) {
        const int ch = base << l, h = H >> l, w = W >> l;
        act(h, w, cb + ch);
        act(h, w, ch);
        act(h, w, ch);
        cb = ch;
    }
    int rc = PAT_OK;
    for (Act& a : u->acts) {
        const size_t n = size_t(max_batch) * a.H * a.W * a.C;
        if (rc == PAT_OK) rc = dalloc(u, &a.y, n);
        if (rc == PAT_OK) rc = dalloc(u, &a.g, n);
    }
    for (int l = 0; l < levels - 1 && rc == PAT_OK; ++l) {
        unsigned char* p = nullptr;
        rc = dalloc(u, &p, size_t(max_batch) * (H >> (l + 1)) * (W >> (l + 1)) * (base << l));
        u->pidx.push_back(p);
    }
    // scratch: the largest im2col (and its transpose) over all convolutions, forward and data gradient
    size_t colmax = 0, wtmax = 0, dtmax = 0;
    for (const Conv& c : u->convs) {
        const size_t P = size_t(max_batch) * c.H * c.W;
        colmax = std::max(colmax, P * size_t(c.k * c.k) * std::max(c.cin, c.cout));
        wtmax = std::max(wtmax, c.nw());
        dtmax = std::max(dtmax, P * size_t(std::max(c.cout, 8)));
    }
    u->col_elems = colmax;
    if (rc == PAT_OK) rc = dalloc(u, &u->col, colmax);
    if (rc == PAT_OK) rc = dalloc(u, &u->colt, colmax);
    if (rc == PAT_OK) rc = dalloc(u, &u->dt, dtmax);
    if (rc == PAT_OK) rc = dalloc(u, &u->wt, std::max<size_t>(wtmax, 8 * 64));
    if (rc == PAT_OK) rc = dalloc(u, &u->param, u->nparam);
    if (rc == PAT_OK) rc = dalloc(u, &u->grad, u->nparam);
    if (rc == PAT_OK) rc = dalloc(u, &u->m, u->nparam);
    if (rc == PAT_OK) rc = dalloc(u, &u->v, u->nparam);
    if (rc == PAT_OK) rc = dalloc(u, &u->wbf, u->nweight_bf);
    if (rc == PAT_OK) rc = dalloc(u, &u->out, size_t(max_batch) * H * W);
    if (rc == PAT_OK) rc = dalloc(u, &u->part, 256);
    if (rc == PAT_OK) rc = dalloc(u, &u->loss, 1);
    if (rc == PAT_OK) rc = dalloc(u, &u->status, 1);
    if (rc == PAT_OK && cudaMemset(u->status, 0, sizeof(int)) != cudaSuccess) rc = cuda_fail(cudaGetLastError(), "unet status");
    if (rc != PAT_OK) {
        pat_unet_destroy(u);
        return rc;
    }
    *out = u;
    return PAT_OK;
}

extern "C" void pat_unet_destroy(pat_unet u) {
    if (!u) return;
    for (void* p : u->allocs) cudaFree(p);
    delete u;
}

extern "C" size_t pat_unet_param_count(pat_unet u) { return u ? u->nparam : 0; }

extern "C" int pat_unet_param_layout(pat_unet u, int* n_convs, int* h_desc) {
    if (!u || !n_convs) { set_error("pat_unet_param_layout: null argument"); return PAT_EINVAL; }
    *n_convs = int(u->convs.size());
    if (h_desc)
        for (size_t i = 0; i < u->convs.size(); ++i) {
            const Conv& c = u->convs[i];
            int* d = h_desc + 6 * i;
            d[0] = c.cin;
            d[1] = c.cout;
            d[2] = c.k;
            d[3] = int(c.w_off);
            d[4] = int(c.b_off);
            d[5] = c.H;
        }
    return PAT_OK;
}

// refresh the bf16 weight copies from the fp32 parameters
static int sync_bf16(pat_unet_s* u, cudaStream_t st) {
    for (const Conv& c : u->convs) RC(unet_f32_to_bf16(st, u->param + c.w_off, u->wbf + c.wb_off, c.nw()));
    return PAT_OK;
}

extern "C" int pat_unet_set_params(pat_unet u, const float* d_params, void* stream) {
    if (!u || !d_params) { set_error("pat_unet_set_params: null argument"); return PAT_EINVAL; }
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    PAT_CUDA(cudaMemcpyAsync(u->param, d_params, u->nparam * sizeof(float), cudaMemcpyDeviceToDevice, st));
    PAT_CUDA(cudaMemsetAsync(u->m, 0, u->nparam * sizeof(float), st));
    PAT_CUDA(cudaMemsetAsync(u->v, 0, u->nparam * sizeof(float), st));
    u->step = 0;
    return sync_bf16(u, st);
}

extern "C" int pat_unet_get_params(pat_unet u, float* d_params, void* stream) {
    if (!u || !d_params) { set_error("pat_unet_get_params: null argument"); return PAT_EINVAL; }
    PAT_CUDA(cudaMemcpyAsync(d_params, u->param, u->nparam * sizeof(float), cudaMemcpyDeviceToDevice,
                             static_cast<cudaStream_t>(stream)));
    return PAT_OK;
}

extern "C" int pat_unet_forward(pat_unet u, const float* d_in, int B, float* d_out, void* stream) {
    if (!u || !d_in || !d_out) { set_error("pat_unet_forward: null argument"); return PAT_EINVAL; }
    RC(check_batch(u, B));
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    RC(forward(u, st, d_in, B));
    PAT_CUDA(cudaMemcpyAsync(d_out, u->out, size_t(B) * u->H * u->W * sizeof(float), cudaMemcpyDeviceToDevice, st));
    return PAT_OK;
}

// loss and parameter gradients (into the model's gradient buffer, optionally copied to d_grad)
static int loss_and_grads(pat_unet_s* u, cudaStream_t st, const float* d_in, const float* d_target, int B) {
    RC(forward(u, st, d_in, B));
    const size_t P = size_t(B) * u->H * u->W;
    const Act& top = u->acts.back();
    // dL/dout in a bf16 [P][8] buffer (channel 0 used) for the final 1x1 convolution
    __nv_bfloat16* dout = u->dt;
    PAT_CUDA(cudaMemsetAsync(dout, 0, P * 8 * sizeof(__nv_bfloat16), st));
    RC(unet_mse(st, u->out, d_target, dout, P, 8, u->part, u->loss));
    // final conv (1x1, cin -> 1): gradients by GEMMs on [P][8] operands
    const Conv& c = u->convs.back();
    float* dW = u->grad + c.w_off;
    float* db = u->grad + c.b_off;
    // bias: db = sum_p dout[p][0]
    RC(unet_bias_grad(st, dout, db, P, 1, 8));
    // the output gradient is copied out before the weight-gradient transposes reuse the scratch
    __nv_bfloat16* doutc = u->colt;
    PAT_CUDA(cudaMemcpyAsync(doutc, dout, P * 8 * sizeof(__nv_bfloat16), cudaMemcpyDeviceToDevice, st));
    // dW[0][ci] = sum_p dout[p] top[p][ci]: transposes [8][P] and [cin][P]
    RC(unet_transpose(st, doutc, u->dt, int(P), 8, 8));
    RC(unet_transpose(st, top.y, u->col, int(P), c.cin, c.cin));
    PAT_CUDA(cudaMemsetAsync(dW, 0, c.nw() * sizeof(float), st));
    {
        const int splitk = std::max(1, std::min(64, int(P / 4096)));
        // rows 1..7 of the transposed output gradient are zero; only row 0 (= dW) is kept
        RC(net_gemm(u, st, u->dt, int(P), u->col, int(P), 1, c.cin, int(P), nullptr, 0, dW, c.cin, 2, splitk));
    }
    // data gradient of the final conv: dtop[p][ci] = dout[p] W[ci]: GEMM with K = 8 (W padded)
    __nv_bfloat16* wpad = u->wt;
    PAT_CUDA(cudaMemsetAsync(wpad, 0, size_t(c.cin) * 8 * sizeof(__nv_bfloat16), st));
    RC(unet_copy_ch(st, u->wbf + c.wb_off, wpad, size_t(c.cin), 1, 1, 8, 0));
    RC(net_gemm(u, st, doutc, 8, wpad, 8, int(P), c.cin, 8, nullptr, 0, top.g, c.cin, 0, 1));
    // the rest of the network
    Layout L = layout_of(u);
    auto& A = u->acts;
    int ci = int(u->convs.size()) - 2;
    for (int d = u->levels - 2; d >= 0; --d) {
        const Act& cat = A[L.dec_cat[d]];
        const Act& da = A[L.dec_a[d]];
        const Act& db2 = A[L.dec_b[d]];
        const size_t Pl = size_t(B) * db2.H * db2.W;
        RC(unet_relu_bwd(st, db2.g, db2.y, Pl * db2.C));
        RC(conv_bwd(u, st, u->convs[ci--], da.y, da.C, B, db2.g, da.g));
        RC(unet_relu_bwd(st, da.g, da.y, Pl * da.C));
        RC(conv_bwd(u, st, u->convs[ci--], cat.y, cat.C, B, da.g, cat.g));
        const Act& below = (d == 0) ? A[L.enc_b.back()] : A[L.dec_b[d - 1]];
        RC(unet_upsample_bwd(st, cat.g, below.g, B, below.H, below.W, below.C, cat.C, 0));
    }
    for (int l = u->levels - 1; l >= 0; --l) {
        const Act& ea = A[L.enc_a[l]];
        const Act& eb = A[L.enc_b[l]];
        const size_t Pl = size_t(B) * eb.H * eb.W;
        if (l < u->levels - 1) {
            const Act& pa = A[L.pool[l]];
            RC(unet_maxpool_bwd(st, pa.g, u->pidx[l], eb.g, B, eb.H, eb.W, eb.C));
            const int d = u->levels - 2 - l;
            const Act& cat = A[L.dec_cat[d]];
            const int below_c = (d == 0) ? A[L.enc_b.back()].C : A[L.dec_b[d - 1]].C;
            RC(unet_add_ch(st, eb.g, cat.g, Pl, eb.C, cat.C, below_c));
        }
        RC(unet_relu_bwd(st, eb.g, eb.y, Pl * eb.C));
        RC(conv_bwd(u, st, u->convs[2 * l + 1], ea.y, ea.C, B, eb.g, ea.g));
        RC(unet_relu_bwd(st, ea.g, ea.y, Pl * ea.C));
        const Act& in = (l == 0) ? A[L.input] : A[L.pool[l - 1]];
        RC(conv_bwd(u, st, u->convs[2 * l], in.y, in.C, B, ea.g, l == 0 ? nullptr : in.g));
    }
    return PAT_OK;
}

extern "C" int pat_unet_grads(pat_unet u, const float* d_in, const float* d_target, int B, float* d_grad,
                              double* d_loss, void* stream) {
    if (!u || !d_in || !d_target) { set_error("pat_unet_grads: null argument"); return PAT_EINVAL; }
    RC(check_batch(u, B));
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    RC(loss_and_grads(u, st, d_in, d_target, B));
    if (d_grad) PAT_CUDA(cudaMemcpyAsync(d_grad, u->grad, u->nparam * sizeof(float), cudaMemcpyDeviceToDevice, st));
    if (d_loss) PAT_CUDA(cudaMemcpyAsync(d_loss, u->loss, sizeof(double), cudaMemcpyDeviceToDevice, st));
    return PAT_OK;
}

extern "C" int pat_unet_train_step(pat_unet u, const float* d_in, const float* d_target, int B, float lr,
                                   double* d_loss, void* stream) {
    if (!u || !d_in || !d_target) { set_error("pat_unet_train_step: null argument"); return PAT_EINVAL; }
    RC(check_batch(u, B));
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    RC(loss_and_grads(u, st, d_in, d_target, B));
    ++u->step;
    const float b1 = 0.9f, b2 = 0.999f;
    const float bc1 = 1.f - std::pow(b1, float(u->step)), bc2 = 1.f - std::pow(b2, float(u->step));
    RC(unet_adam(st, u->param, nullptr, u->grad, u->m, u->v, u->nparam, lr, b1, b2, 1e-8f, bc1, bc2));
    RC(sync_bf16(u, st));
    if (d_loss) PAT_CUDA(cudaMemcpyAsync(d_loss, u->loss, sizeof(double), cudaMemcpyDeviceToDevice, st));
    return PAT_OK;
}

extern "C" int pat_unet_set_gemm_path(pat_unet u, int path) {
    if (!u || path < 0 || path > 1) { set_error("pat_unet_set_gemm_path: null network or path not 0/1"); return PAT_EINVAL; }
    u->gemm_path = path;
    return PAT_OK;
}

extern "C" int pat_unet_status(pat_unet u, int* h_flag, void* stream) {
    if (!u || !h_flag) { set_error("pat_unet_status: null argument"); return PAT_EINVAL; }
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    int f = 0;
    PAT_CUDA(cudaMemcpyAsync(&f, u->status, sizeof(int), cudaMemcpyDeviceToHost, st));
    PAT_CUDA(cudaStreamSynchronize(st));
    *h_flag = f & PAT_STATUS_TC05;
    return PAT_OK;
}

extern "C" int pat_gemm_bf16(const void* d_A, int lda, const void* d_B, int ldb, int M, int N, int K, float* d_C,
                             int ldc, int path, int* d_status, void* stream) {
    if (!d_A || !d_B || !d_C || M < 1 || N < 1 || K < 1 || ldc < N || lda < K || ldb < K || path < 0 || path > 1) {
        set_error("pat_gemm_bf16: null buffer, size < 1, pitch below the row length or path not 0/1");
        return PAT_EINVAL;
    }
    const auto* A = static_cast<const __nv_bfloat16*>(d_A);
    const auto* B = static_cast<const __nv_bfloat16*>(d_B);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    if (path == 1) {
        if (!unet_gemm_tc05_supported(A, lda, B, ldb, M, N, K)) {
            set_error("pat_gemm_bf16: the tcgen05 path needs K >= 64, pitches that are multiples of 8 and 16-byte "
                      "aligned operands");
            return PAT_EINVAL;
        }
        return unet_gemm_tc05(st, A, lda, B, ldb, M, N, K, nullptr, 0, d_C, ldc, 1, 1, d_status);
    }
    return unet_gemm(st, A, lda, B, ldb, M, N, K, nullptr, 0, d_C, ldc, 1, 1);
}

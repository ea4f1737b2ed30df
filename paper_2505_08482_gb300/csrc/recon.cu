// pat_reconstruct: projected L-BFGS with backtracking (Sec. 3, Eq.
// BFGS_iterations, Algorithm 1, Eq. bound_constraints) over the
// coarse-to-fine multigrid schedule (Sec. 3.1, data interpolated in time to
// every level as in Sec. 4.1.2).
//
// Vectors live on the device in FP32 (block-scaled variables z = x / sigma);
// dot products accumulate in FP64 and the line-search and pair-acceptance
// decisions are taken on the host in FP64.  The two-loop recursion keeps its
// scalars (rho_j, lambda_j, beta, H0) in device memory, so it needs no host
// round trip.  Readings where the paper is silent: H0 from the newest pair
// (alpha0 / ||g||_inf without pairs); direction components leaving the box at
// an active bound are zeroed; Armijo backtracking by halving from alpha = 1
// with memory reset and one steepest-descent retry on failure; pairs kept
// only if s^T y > 1e-10 ||s|| ||y||; a level stops after `iters` iterations
// or when the relative decrease of J falls below rtol.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <vector>

#include "pat_internal.h"
#include "vec.h"

using namespace pat;

namespace {

#define RC(x)                          \
    do {                               \
        int rc_ = (x);                 \
        if (rc_ != PAT_OK) return rc_; \
    } while (0)

struct DevScalars {
    double* part;   // [kPartials]
    double* tmp;    // scratch scalars [8]
    double* lam;    // [mem]
    double* rho;    // [mem]
    double* beta;   // [1]
    double* h0;     // [1]
    double* J;      // [1]
};

struct Level {
    cudaStream_t st;
    size_t V, n0;
    Box box;
    float *x, *z, *g, *d, *xt, *zt, *gt, *graw, *q, *psi;
    std::vector<float*> S, Y;   // ring of pairs
    DevScalars sc;
};

int read_scalar(cudaStream_t st, const double* d, double* h) {
    PAT_CUDA(cudaMemcpyAsync(h, d, sizeof(double), cudaMemcpyDeviceToHost, st));
    PAT_CUDA(cudaStreamSynchronize(st));
    return PAT_OK;
}

int host_dot(Level& L, const float* a, const float* b, double* out) {
    RC(vdot(L.st, a, b, L.V, L.sc.tmp, L.sc.part));
    return read_scalar(L.st, L.sc.tmp, out);
}

class Recon {
public:
    Recon(const pat_recon_cfg& c, cudaStream_t st) : cfg(c), st(st) {}
    int run(const float* ymeas, const float* w, float* c_io, float* p0_io, pat_report* rep);

private:
    const pat_recon_cfg& cfg;
    cudaStream_t st;
    std::vector<void*> allocs;

    template <class T>
    int alloc(T** p, size_t n) {
        void* v = nullptr;
        PAT_CUDA(cudaMallocAsync(&v, std::max<size_t>(n * sizeof(T), 256), st));
        allocs.push_back(v);
        *p = static_cast<T*>(v);
        return PAT_OK;
    }

public:
    void free_all() {
        for (void* v : allocs) cudaFreeAsync(v, st);
        allocs.clear();
    }
};

int steepest(Level& L, double alpha0) {
    double gi = 0.0;
    RC(vabsmax(L.st, L.g, L.V, L.sc.tmp, L.sc.part));
    RC(read_scalar(L.st, L.sc.tmp, &gi));
    const float a = gi > 0 ? float(-alpha0 / gi) : 0.f;
    return vaxpby(L.st, L.d, a, L.g, 0.f, nullptr, L.V);
}

// d = -H g with the pairs in order oldest .. newest (indices into the ring)
int two_loop(Level& L, const std::vector<int>& order) {
    RC(vaxpby(L.st, L.q, 1.f, L.g, 0.f, nullptr, L.V));
    for (int t = int(order.size()) - 1; t >= 0; --t) {
        const int j = order[t];
        RC(vdot(L.st, L.S[j], L.q, L.V, L.sc.lam + j, L.sc.part, L.sc.rho + j, 1.0));
        RC(vaxpy_dev(L.st, L.q, L.Y[j], L.V, L.sc.lam + j, nullptr, -1.f));
    }
    RC(vscale_dev(L.st, L.psi, L.q, L.V, L.sc.h0, 1.f));
    for (size_t t = 0; t < order.size(); ++t) {
        const int j = order[t];
        RC(vdot(L.st, L.Y[j], L.psi, L.V, L.sc.beta, L.sc.part, L.sc.rho + j, 1.0));
        RC(vaxpy_dev(L.st, L.psi, L.S[j], L.V, L.sc.lam + j, L.sc.beta, 1.f));
    }
    return vaxpby(L.st, L.d, -1.f, L.psi, 0.f, nullptr, L.V);
}

int Recon::run(const float* ymeas, const float* w, float* c_io, float* p0_io, pat_report* rep) {
    const int K = cfg.K, M = cfg.m;
    const int Nf = cfg.levels[cfg.nlevels - 1];
    const double T = (cfg.nt_data - 1) * cfg.dt_data;
    const double sc = (cfg.c_hi - cfg.c_lo) / 4.0, sp = cfg.sigma_p0;
    const int memsz = std::max(cfg.mem, 1);
    auto t_start = std::chrono::steady_clock::now();
    if (rep) {
        rep->count = 0;
        rep->status = PAT_OK;
        rep->total_ms = 0;
    }
    // initial guess on the finest grid, stacked [K+1][Nf][Nf]
    float* xf;
    RC(alloc(&xf, size_t(K + 1) * Nf * Nf));
    PAT_CUDA(cudaMemcpyAsync(xf, p0_io, size_t(K) * Nf * Nf * sizeof(float), cudaMemcpyDeviceToDevice, st));
    PAT_CUDA(cudaMemcpyAsync(xf + size_t(K) * Nf * Nf, c_io, size_t(Nf) * Nf * sizeof(float),
                             cudaMemcpyDeviceToDevice, st));
    float* xprev = xf;
    int nprev = Nf;
    for (int li = 0; li < cfg.nlevels; ++li) {
        const int N = cfg.levels[li];
        pat_grid g{};
        g.n = N;
        g.pml = pat_pml_auto(N, cfg.min_pml);
        if (g.pml < 0) { set_error("pat_reconstruct: no valid PML for level side %d", N); return PAT_EINVAL; }
        g.dx = cfg.L / N;
        g.dt = cfg.cfl * g.dx / cfg.c_hi;
        g.nt = int(std::lround(T / g.dt)) + 1;
        g.c_ref = cfg.c_hi;
        g.rho0 = cfg.rho0;
        g.pml_alpha = cfg.pml_alpha;
        g.c_bg = cfg.c_bg;
        pat_plan plan = nullptr;
        RC(pat_plan_create(&plan, &g, M, cfg.h_sensor_xy, K, cfg.ckpt_every));
        struct PlanGuard { pat_plan p; ~PlanGuard() { pat_plan_destroy(p); } } guard{plan};
        const size_t wsb = pat_workspace_bytes(plan, PAT_WS_GRADIENT);
        void* ws;
        RC(alloc(reinterpret_cast<char**>(&ws), wsb));
        float* yl;
        RC(alloc(&yl, size_t(K) * g.nt * M));
        RC(vtime_interp(st, ymeas, yl, K, cfg.nt_data, g.nt, M, cfg.dt_data, g.dt));

        Level L;
        L.st = st;
        L.V = size_t(K + 1) * N * N;
        L.n0 = size_t(K) * N * N;
        L.box = Box{float(cfg.p0_lo / sp), INFINITY, float(sp), float(cfg.c_lo / sc), float(cfg.c_hi / sc),
                    float(sc)};
        float** vecs[] = {&L.x, &L.z, &L.g, &L.d, &L.xt, &L.zt, &L.gt, &L.graw, &L.q, &L.psi};
        for (float** v : vecs) RC(alloc(v, L.V));
        L.S.resize(memsz);
        L.Y.resize(memsz);
        for (int j = 0; j < memsz; ++j) {
            RC(alloc(&L.S[j], L.V));
            RC(alloc(&L.Y[j], L.V));
        }
        RC(alloc(&L.sc.part, kPartials));
        RC(alloc(&L.sc.tmp, 8));
        RC(alloc(&L.sc.lam, memsz));
        RC(alloc(&L.sc.rho, memsz));
        RC(alloc(&L.sc.beta, 1));
        RC(alloc(&L.sc.h0, 1));
        RC(alloc(&L.sc.J, 1));
        // x0 = resample of the previous level (or of the initial guess); z = P(x0 / sigma)
        RC(vresample(st, xprev, L.xt, K + 1, nprev, N));
        RC(vblockscale(st, L.zt, L.xt, L.V, L.n0, float(sp), float(sc), 1));
        RC(vproject(st, L.z, L.x, L.zt, L.zt, 0.f, L.V, L.n0, L.box));
        const float* xc = L.x + L.n0;   // c block
        auto grad_at = [&](const float* xv, float* graw, float* gscaled, double* J) -> int {
            RC(pat_adjoint_grad(plan, xv + L.n0, xv, yl, w, graw, graw + L.n0, L.sc.J, nullptr, ws, wsb, st));
            RC(vblockscale(st, gscaled, graw, L.V, L.n0, float(sp), float(sc), 0));
            return read_scalar(st, L.sc.J, J);
        };
        (void)xc;
        double J;
        RC(grad_at(L.x, L.graw, L.g, &J));
        std::vector<int> order;   // ring indices, oldest first
        int next_slot = 0;
        bool have_h0 = false;
        for (int it = 0; it < cfg.iters; ++it) {
            auto t0 = std::chrono::steady_clock::now();
            if (!order.empty()) {
                RC(two_loop(L, cfg.mem > 0 ? order : std::vector<int>()));
            } else if (have_h0) {
                RC(vscale_dev(st, L.d, L.g, L.V, L.sc.h0, -1.f));
            } else {
                RC(steepest(L, cfg.alpha0));
            }
            RC(vclip_dir(st, L.d, L.z, L.V, L.n0, L.box));
            double gd;
            RC(host_dot(L, L.g, L.d, &gd));
            if (gd >= 0.0) {
                order.clear();
                RC(steepest(L, cfg.alpha0));
                RC(vclip_dir(st, L.d, L.z, L.V, L.n0, L.box));
            }
            bool accepted = false, tried_reset = false;
            int trials = 0;
            double alpha = 1.0, Jt = 0.0;
            for (;;) {
                alpha = 1.0;
                for (int h = 0; h <= cfg.max_halvings; ++h) {
                    RC(vproject(st, L.zt, L.xt, L.z, L.d, float(alpha), L.V, L.n0, L.box));
                    RC(objective(plan, L.xt + L.n0, L.xt, yl, w, L.sc.J, ws, wsb, st));
                    RC(read_scalar(st, L.sc.J, &Jt));
                    ++trials;
                    RC(vaxpby(st, L.q, 1.f, L.zt, -1.f, L.z, L.V));
                    double dec;
                    RC(host_dot(L, L.g, L.q, &dec));
                    if (std::isfinite(Jt) && Jt <= J + cfg.c1 * dec) {
                        accepted = true;
                        break;
                    }
                    alpha *= 0.5;
                }
                if (accepted || tried_reset) break;
                tried_reset = true;
                order.clear();
                have_h0 = false;
                RC(steepest(L, cfg.alpha0));
                RC(vclip_dir(st, L.d, L.z, L.V, L.n0, L.box));
            }
            double gn2;
            RC(host_dot(L, L.g, L.g, &gn2));
            auto ms = [&]() {
                return std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
            };
            if (!accepted) {
                if (rep) {
                    if (rep->count < rep->capacity && rep->iters)
                        rep->iters[rep->count++] = pat_iter_report{li, it, J, std::sqrt(gn2), 0.0, trials, J, ms()};
                    rep->status = PAT_ELINESEARCH;
                }
                break;
            }
            double Jn;
            RC(grad_at(L.xt, L.graw, L.gt, &Jn));
            // pair (s, y) into the next ring slot
            const int slot = next_slot;
            RC(vaxpby(st, L.S[slot], 1.f, L.zt, -1.f, L.z, L.V));
            RC(vaxpby(st, L.Y[slot], 1.f, L.gt, -1.f, L.g, L.V));
            double sy, ss, yy;
            RC(host_dot(L, L.S[slot], L.Y[slot], &sy));
            RC(host_dot(L, L.S[slot], L.S[slot], &ss));
            RC(host_dot(L, L.Y[slot], L.Y[slot], &yy));
            if (sy > 1e-10 * std::sqrt(ss) * std::sqrt(yy)) {
                const double rho = 1.0 / sy, h0 = sy / yy;
                PAT_CUDA(cudaMemcpy(L.sc.rho + slot, &rho, sizeof(double), cudaMemcpyHostToDevice));
                PAT_CUDA(cudaMemcpy(L.sc.h0, &h0, sizeof(double), cudaMemcpyHostToDevice));
                have_h0 = true;
                if (cfg.mem > 0) {
                    order.erase(std::remove(order.begin(), order.end(), slot), order.end());
                    order.push_back(slot);
                    if (int(order.size()) > cfg.mem) order.erase(order.begin());
                    next_slot = (slot + 1) % memsz;
                } else {
                    order.clear();
                }
            }
            if (rep && rep->count < rep->capacity && rep->iters)
                rep->iters[rep->count++] = pat_iter_report{li, it, J, std::sqrt(gn2), alpha, trials, Jn, ms()};
            const double rel = J > 0 ? (J - Jn) / J : 0.0;
            std::swap(L.z, L.zt);
            std::swap(L.x, L.xt);
            std::swap(L.g, L.gt);
            J = Jn;
            if (rel < cfg.rtol) break;
        }
        xprev = L.x;
        nprev = N;
    }
    // result on the finest level (levels end at Nf)
    PAT_CUDA(cudaMemcpyAsync(p0_io, xprev, size_t(K) * Nf * Nf * sizeof(float), cudaMemcpyDeviceToDevice, st));
    PAT_CUDA(cudaMemcpyAsync(c_io, xprev + size_t(K) * Nf * Nf, size_t(Nf) * Nf * sizeof(float),
                             cudaMemcpyDeviceToDevice, st));
    PAT_CUDA(cudaStreamSynchronize(st));
    if (rep)
        rep->total_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t_start).count();
    return PAT_OK;
}

}  // namespace

extern "C" int pat_reconstruct(const pat_recon_cfg* cfg, const float* y_meas, const float* w, float* c_io,
                               float* p0_io, pat_report* rep, void* stream) {
    if (!cfg || !y_meas || !w || !c_io || !p0_io) { set_error("pat_reconstruct: null argument"); return PAT_EINVAL; }
    if (cfg->nlevels < 1 || !cfg->levels || cfg->K < 1 || cfg->m < 1 || !cfg->h_sensor_xy || cfg->nt_data < 1 ||
        !(cfg->dt_data > 0) || !(cfg->L > 0) || !(cfg->cfl > 0) || !(cfg->c_hi > cfg->c_lo) || cfg->mem < 0 ||
        cfg->iters < 0 || cfg->max_halvings < 0 || cfg->ckpt_every < 1 || !(cfg->sigma_p0 > 0) ||
        !(cfg->alpha0 > 0)) {
        set_error("pat_reconstruct: invalid configuration");
        return PAT_EINVAL;
    }
    for (int i = 0; i < cfg->nlevels; ++i)
        if (cfg->levels[i] < 2) { set_error("pat_reconstruct: level side < 2"); return PAT_EINVAL; }
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    Recon r(*cfg, st);
    int rc = r.run(y_meas, w, c_io, p0_io, rep);
    r.free_all();
    cudaError_t e = cudaStreamSynchronize(st);
    if (rc == PAT_OK && e != cudaSuccess) rc = cuda_fail(e, "pat_reconstruct");
    return rc;
}

// pat_reconstruct / pat_reconstruct_batched: projected L-BFGS with
// backtracking (Sec. 3, Eq. BFGS_iterations, Algorithm 1, Eq.
// bound_constraints) over the coarse-to-fine multigrid schedule (Sec. 3.1,
// data interpolated in time to every level as in Sec. 4.1.2).
//
// A call reconstructs one or several independent instances that share the
// grid levels, the sensors and the time grid.  Every objective or gradient
// evaluation is one batched solve over all instances (one launch per pass);
// each instance keeps its own iterate, gradient, curvature pairs and FP64 line
// search, and the instances advance in lockstep: a line-search round
// evaluates the trial points of all instances still searching, an instance
// that has accepted its step keeps its point.
//
// Vectors live on the device in FP32 (block-scaled variables z = x / sigma,
// one contiguous vector [p0_1..p0_K, c] per instance); dot products
// accumulate in FP64 into device scalars that are read back once per phase.
// Readings where the paper is silent: H0 from the newest pair (alpha0 /
// ||g||_inf without pairs); direction components leaving the box at an
// active bound are zeroed; Armijo backtracking by halving from alpha = 1 with
// memory reset and one steepest-descent retry on failure; pairs kept only if
// s^T y > 1e-10 ||s|| ||y||; an instance stops after `iters` iterations per
// level or when the relative decrease of its J falls below rtol.
#include <cuda_runtime.h>

#include <cstdio>

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

using Clock = std::chrono::steady_clock;
double ms_since(Clock::time_point t) { return std::chrono::duration<double, std::milli>(Clock::now() - t).count(); }

// scalar slots per instance in the device scalar array
enum { S_GD, S_DEC, S_GG, S_SY, S_SS, S_YY, S_MAX, S_BETA, S_H0, S_EC, S_CT, S_EP, S_PT, S_COUNT };

struct Inst {
    int K;
    size_t V, n0;               // vector length, length of the p0 block
    float *x, *z, *g, *d, *xt, *zt, *gt, *q, *psi;
    float* ct = nullptr;        // true c resampled to the level (E_c tracking), or null
    float* pt = nullptr;        // true p0 (all K) resampled to the level (E_p0 tracking), or null
    float* zp = nullptr;        // Xi^{-1} (x - eta) at the accepted point x (the prior solves' warm start)
    float* zpt = nullptr;       // the same at the trial point xt
    bool zp_warm = false;
    std::vector<float*> S, Y;   // ring of curvature pairs
    double* lam;                // [mem] device
    double* rho;                // [mem] device
    std::vector<int> order;     // ring slots, oldest first
    int next_slot = 0;
    bool have_h0 = false;
    double J = 0, Jt = 0;
    bool active = true;         // still iterating on this level
    bool done = false;          // finished every level
    double finish_ms = 0;
    // line search state
    double alpha = 1;
    bool accepted = false, tried_reset = false, failed = false;
    int trials = 0;
    Clock::time_point t_iter;
};

class Batch {
public:
    Batch(const pat_recon_cfg& c, int ninst, const pat_instance* in, cudaStream_t st)
        : cfg(c), ni(ninst), ins(in), st(st) {}
    ~Batch() {
        for (void* v : allocs) cudaFreeAsync(v, st);
        if (prior) pat_prior_destroy(prior);
    }
    int run();

private:
    const pat_recon_cfg& cfg;
    int ni;
    const pat_instance* ins;
    cudaStream_t st;
    std::vector<void*> allocs;
    std::vector<Inst> I;
    Box box{};
    double* dsc = nullptr;          // [ni][S_COUNT] device scalars
    std::vector<double> hsc;        // host copy
    double* part = nullptr;         // [kPartials]
    double* dJ = nullptr;           // [ni] batched J
    std::vector<double> hJ;
    // batched plan buffers of the current level
    pat_plan plan = nullptr;
    pat_prior prior = nullptr;      // prior terms on the current level (null: data term only)
    void* ws = nullptr;
    size_t wsb = 0;
    float *bp0 = nullptr, *bc = nullptr, *bgp0 = nullptr, *bgc = nullptr, *bym = nullptr, *bw = nullptr;
    int Ktot = 0, N = 0;
    Clock::time_point t0;

    template <class T>
    int alloc(T** p, size_t n) {
        void* v = nullptr;
        PAT_CUDA(cudaMallocAsync(&v, std::max<size_t>(n * sizeof(T), 256), st));
        allocs.push_back(v);
        *p = static_cast<T*>(v);
        return PAT_OK;
    }
    int sync_scalars() {
        PAT_CUDA(cudaMemcpyAsync(hsc.data(), dsc, hsc.size() * sizeof(double), cudaMemcpyDeviceToHost, st));
        PAT_CUDA(cudaStreamSynchronize(st));
        return PAT_OK;
    }
    double* sc(int i, int s) { return dsc + size_t(i) * S_COUNT + s; }
    double hs(int i, int s) const { return hsc[size_t(i) * S_COUNT + s]; }
    int set_scalar(int i, int s, double v) {
        hsc[size_t(i) * S_COUNT + s] = v;
        PAT_CUDA(cudaMemcpyAsync(sc(i, s), &hsc[size_t(i) * S_COUNT + s], sizeof(double), cudaMemcpyHostToDevice,
                                 st));
        return PAT_OK;
    }
    int level(int li, const float* const* xprev, int nprev);
    int evaluate(bool grad, bool trial);
    int steepest_all(const std::vector<int>& which);
    int two_loop(Inst& s, int i);
};

// gather the instances' iterates (trial or current) into the batched buffers, run
// the batched objective (or gradient) and scatter J (and the scaled gradients) back
int Batch::evaluate(bool grad, bool trial) {
    size_t ok = 0;
    const size_t nn = size_t(N) * N;
    for (int i = 0; i < ni; ++i) {
        const Inst& s = I[i];
        const float* x = trial ? s.xt : s.x;
        PAT_CUDA(cudaMemcpyAsync(bp0 + ok * nn, x, s.n0 * sizeof(float), cudaMemcpyDeviceToDevice, st));
        PAT_CUDA(cudaMemcpyAsync(bc + size_t(i) * nn, x + s.n0, nn * sizeof(float), cudaMemcpyDeviceToDevice, st));
        ok += s.K;
    }
    if (grad) {
        RC(pat_adjoint_grad(plan, bc, bp0, bym, bw, bgp0, bgc, dJ, nullptr, ws, wsb, st));
        ok = 0;
        const float sp = float(cfg.sigma_p0), scs = float((cfg.c_hi - cfg.c_lo) / 4.0);
        for (int i = 0; i < ni; ++i) {
            Inst& s = I[i];
            float* gdst = trial ? s.gt : s.g;
            RC(vblockscale(st, gdst, bgp0 + ok * nn, s.n0, s.n0, sp, sp, 0));
            RC(vblockscale(st, gdst + s.n0, bgc + size_t(i) * nn, nn, 0, scs, scs, 0));
            ok += s.K;
        }
    } else {
        RC(objective(plan, bc, bp0, bym, bw, dJ, ws, wsb, st));
    }
    if (prior) {   // prior terms of Eq. Minimised_functional: into J and the block-scaled gradient
        const double sp = cfg.sigma_p0, scs = (cfg.c_hi - cfg.c_lo) / 4.0;
        for (int i = 0; i < ni; ++i) {
            Inst& s = I[i];
            std::vector<double> eta(s.K + 1, cfg.prior_eta_p0), sig(s.K + 1, cfg.prior_sigma_p0), gs(s.K + 1, sp);
            eta[s.K] = cfg.prior_eta_c;
            sig[s.K] = cfg.prior_sigma_c;
            gs[s.K] = scs;
            float* gdst = grad ? (trial ? s.gt : s.g) : nullptr;
            // every solve starts from the accepted point's solution, so that an instance's
            // results do not depend on evaluations made for other instances of a batch
            float* zdst = trial ? s.zpt : s.zp;
            if (trial && s.zp_warm)
                PAT_CUDA(cudaMemcpyAsync(s.zpt, s.zp, s.V * sizeof(float), cudaMemcpyDeviceToDevice, st));
            RC(pat_prior_eval(prior, trial ? s.xt : s.x, s.K + 1, eta.data(), sig.data(), gs.data(), zdst, gdst,
                              dJ + i, 1e-5, 500, s.zp_warm ? 1 : 0, nullptr, st));
            if (!trial) s.zp_warm = true;
        }
    }
    PAT_CUDA(cudaMemcpyAsync(hJ.data(), dJ, ni * sizeof(double), cudaMemcpyDeviceToHost, st));
    PAT_CUDA(cudaStreamSynchronize(st));
    return PAT_OK;
}

int Batch::steepest_all(const std::vector<int>& which) {
    for (int i : which) RC(vabsmax(st, I[i].g, I[i].V, sc(i, S_MAX), part));
    RC(sync_scalars());
    for (int i : which) {
        const double gi = hs(i, S_MAX);
        RC(vaxpby(st, I[i].d, gi > 0 ? float(-cfg.alpha0 / gi) : 0.f, I[i].g, 0.f, nullptr, I[i].V));
        RC(vclip_dir(st, I[i].d, I[i].z, I[i].V, I[i].n0, box));
    }
    return PAT_OK;
}

// d = -H g with the pairs in order oldest .. newest
int Batch::two_loop(Inst& s, int i) {
    RC(vaxpby(st, s.q, 1.f, s.g, 0.f, nullptr, s.V));
    for (int t = int(s.order.size()) - 1; t >= 0; --t) {
        const int j = s.order[t];
        RC(vdot(st, s.S[j], s.q, s.V, s.lam + j, part, s.rho + j, 1.0));
        RC(vaxpy_dev(st, s.q, s.Y[j], s.V, s.lam + j, nullptr, -1.f));
    }
    RC(vscale_dev(st, s.psi, s.q, s.V, sc(i, S_H0), 1.f));
    for (size_t t = 0; t < s.order.size(); ++t) {
        const int j = s.order[t];
        RC(vdot(st, s.Y[j], s.psi, s.V, sc(i, S_BETA), part, s.rho + j, 1.0));
        RC(vaxpy_dev(st, s.psi, s.S[j], s.V, s.lam + j, sc(i, S_BETA), 1.f));
    }
    return vaxpby(st, s.d, -1.f, s.psi, 0.f, nullptr, s.V);
}

int Batch::level(int li, const float* const* xprev, int nprev) {
    const int M = cfg.m;
    N = cfg.levels[li];
    const double T = (cfg.nt_data - 1) * cfg.dt_data;
    const double sc_c = (cfg.c_hi - cfg.c_lo) / 4.0, sp = cfg.sigma_p0;
    const int memsz = std::max(cfg.mem, 1);
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
    std::vector<int> Ks(ni);
    Ktot = 0;
    for (int i = 0; i < ni; ++i) {
        Ks[i] = ins[i].K;
        Ktot += ins[i].K;
    }
    if (plan) pat_plan_destroy(plan);
    plan = nullptr;
    RC(pat_plan_create_batched(&plan, &g, M, cfg.h_sensor_xy, ni, Ks.data(), cfg.ckpt_every));
    wsb = pat_workspace_bytes(plan, PAT_WS_GRADIENT);
    RC(alloc(reinterpret_cast<char**>(&ws), wsb));
    // forward-step timing (a short run on the forward part of the workspace): the gradient
    // timing of six whole evaluations per level would cost more than it saves here
    if (cfg.autotune) RC(pat_plan_autotune(plan, ws, pat_workspace_bytes(plan, PAT_WS_FORWARD), nullptr, st));
    if (cfg.persistent && pat_plan_set_persistent(plan, 1) != PAT_OK) pat_plan_set_persistent(plan, 0);
    if (prior) pat_prior_destroy(prior);
    prior = nullptr;
    if (cfg.prior_tau > 0) {
        int kmax = 0;
        for (int i = 0; i < ni; ++i) kmax = std::max(kmax, ins[i].K);
        RC(pat_prior_create(N, g.dx, cfg.prior_tau, kmax + 1, &prior));
    }
    if (st) RC(pat_plan_set_graphs(plan, 1));   // one graph per evaluation kind on this level
    const size_t nn = size_t(N) * N;
    RC(alloc(&bp0, Ktot * nn));
    RC(alloc(&bc, ni * nn));
    RC(alloc(&bgp0, Ktot * nn));
    RC(alloc(&bgc, ni * nn));
    RC(alloc(&bym, size_t(Ktot) * g.nt * M));
    RC(alloc(&bw, Ktot));
    for (int i = 0, ok = 0; i < ni; ++i) {
        RC(vtime_interp(st, ins[i].d_y_meas, bym + size_t(ok) * g.nt * M, ins[i].K, cfg.nt_data, g.nt, M,
                        cfg.dt_data, g.dt));
        PAT_CUDA(cudaMemcpyAsync(bw + ok, ins[i].d_w, ins[i].K * sizeof(float), cudaMemcpyDeviceToDevice, st));
        ok += ins[i].K;
    }
    box = Box{float(cfg.p0_lo / sp), INFINITY, float(sp), float(cfg.c_lo / sc_c), float(cfg.c_hi / sc_c),
              float(sc_c)};
    I.assign(ni, Inst{});
    for (int i = 0; i < ni; ++i) {
        Inst& s = I[i];
        s.K = ins[i].K;
        s.V = size_t(s.K + 1) * nn;
        s.n0 = size_t(s.K) * nn;
        float** vecs[] = {&s.x, &s.z, &s.g, &s.d, &s.xt, &s.zt, &s.gt, &s.q, &s.psi};
        for (float** v : vecs) RC(alloc(v, s.V));
        s.S.resize(memsz);
        s.Y.resize(memsz);
        for (int j = 0; j < memsz; ++j) {
            RC(alloc(&s.S[j], s.V));
            RC(alloc(&s.Y[j], s.V));
        }
        RC(alloc(&s.lam, memsz));
        RC(alloc(&s.rho, memsz));
        if (prior) {
            RC(alloc(&s.zp, s.V));
            RC(alloc(&s.zpt, s.V));
        }
        // x0 = resample of the previous level (or of the initial guess); z = P(x0 / sigma)
        RC(vresample(st, xprev[i], s.xt, s.K + 1, nprev, N));
        RC(vblockscale(st, s.zt, s.xt, s.V, s.n0, float(sp), float(sc_c), 1));
        RC(vproject(st, s.z, s.x, s.zt, s.zt, 0.f, s.V, s.n0, box));
        if (ins[i].d_c_true) {
            RC(alloc(&s.ct, nn));
            RC(vresample(st, ins[i].d_c_true, s.ct, 1, cfg.levels[cfg.nlevels - 1], N));
            RC(vdot(st, s.ct, s.ct, nn, sc(i, S_CT), part));
        }
        if (ins[i].d_p0_true) {
            RC(alloc(&s.pt, s.n0));
            RC(vresample(st, ins[i].d_p0_true, s.pt, s.K, cfg.levels[cfg.nlevels - 1], N));
            RC(vdot(st, s.pt, s.pt, s.n0, sc(i, S_PT), part));
        }
    }
    RC(evaluate(true, false));
    for (int i = 0; i < ni; ++i) I[i].J = hJ[i];
    for (int it = 0; it < cfg.iters; ++it) {
        std::vector<int> act;
        for (int i = 0; i < ni; ++i)
            if (I[i].active) act.push_back(i);
        if (act.empty()) break;
        // directions
        std::vector<int> steep;
        for (int i : act) {
            Inst& s = I[i];
            s.t_iter = Clock::now();
            if (!s.order.empty())
                RC(two_loop(s, i));
            else if (s.have_h0)
                RC(vscale_dev(st, s.d, s.g, s.V, sc(i, S_H0), -1.f));
            else
                steep.push_back(i);
        }
        RC(steepest_all(steep));
        for (int i : act) {
            RC(vclip_dir(st, I[i].d, I[i].z, I[i].V, I[i].n0, box));
            RC(vdot(st, I[i].g, I[i].d, I[i].V, sc(i, S_GD), part));
        }
        RC(sync_scalars());
        std::vector<int> bad;
        for (int i : act)
            if (hs(i, S_GD) >= 0.0) {
                I[i].order.clear();
                bad.push_back(i);
            }
        RC(steepest_all(bad));
        // lockstep backtracking
        for (int i : act) {
            Inst& s = I[i];
            s.alpha = 1.0;
            s.accepted = s.tried_reset = s.failed = false;
            s.trials = 0;
        }
        for (int round = 0; round < 2; ++round) {
            for (int h = 0; h <= cfg.max_halvings; ++h) {
                std::vector<int> srch;
                for (int i : act)
                    if (!I[i].accepted && !I[i].failed && (round == 0 || I[i].tried_reset)) srch.push_back(i);
                if (srch.empty()) break;
                for (int i = 0; i < ni; ++i) {
                    Inst& s = I[i];
                    bool searching = std::find(srch.begin(), srch.end(), i) != srch.end();
                    if (searching)
                        RC(vproject(st, s.zt, s.xt, s.z, s.d, float(s.alpha), s.V, s.n0, box));
                    else if (!(s.active && s.accepted))
                        PAT_CUDA(cudaMemcpyAsync(s.xt, s.x, s.V * sizeof(float), cudaMemcpyDeviceToDevice, st));
                }
                RC(evaluate(false, true));
                for (int i : srch) {
                    Inst& s = I[i];
                    s.Jt = hJ[i];
                    ++s.trials;
                    RC(vaxpby(st, s.q, 1.f, s.zt, -1.f, s.z, s.V));
                    RC(vdot(st, s.g, s.q, s.V, sc(i, S_DEC), part));
                }
                RC(sync_scalars());
                for (int i : srch) {
                    Inst& s = I[i];
                    if (std::isfinite(s.Jt) && s.Jt <= s.J + cfg.c1 * hs(i, S_DEC))
                        s.accepted = true;
                    else
                        s.alpha *= 0.5;
                }
            }
            // instances whose first search failed: drop the memory, retry once with steepest descent
            std::vector<int> retry;
            for (int i : act) {
                Inst& s = I[i];
                if (s.accepted || s.failed) continue;
                if (round == 0) {
                    s.tried_reset = true;
                    s.order.clear();
                    s.have_h0 = false;
                    s.alpha = 1.0;
                    retry.push_back(i);
                } else {
                    s.failed = true;
                }
            }
            if (retry.empty()) break;
            RC(steepest_all(retry));
        }
        for (int i : act)
            if (!I[i].accepted) I[i].failed = true;
        for (int i : act) RC(vdot(st, I[i].g, I[i].g, I[i].V, sc(i, S_GG), part));
        RC(sync_scalars());
        // failed instances stop on this level
        for (int i : act) {
            Inst& s = I[i];
            if (!s.failed) continue;
            pat_report* rep = ins[i].report;
            if (rep) {
                if (rep->count < rep->capacity && rep->iters)
                    rep->iters[rep->count++] = pat_iter_report{
                        li, it, s.J, std::sqrt(hs(i, S_GG)), 0.0, s.trials, s.J, ms_since(s.t_iter), -1.0, -1.0};
                rep->status = PAT_ELINESEARCH;
            }
            s.active = false;
        }
        // gradients at the accepted points (batched; the others keep their point)
        for (int i = 0; i < ni; ++i) {
            Inst& s = I[i];
            if (!(s.active && s.accepted))
                PAT_CUDA(cudaMemcpyAsync(s.xt, s.x, s.V * sizeof(float), cudaMemcpyDeviceToDevice, st));
        }
        bool any = false;
        for (int i : act) any = any || (I[i].active && I[i].accepted);
        if (!any) break;
        RC(evaluate(true, true));
        for (int i : act) {
            Inst& s = I[i];
            if (!s.active) continue;
            const int slot = s.next_slot;
            RC(vaxpby(st, s.S[slot], 1.f, s.zt, -1.f, s.z, s.V));
            RC(vaxpby(st, s.Y[slot], 1.f, s.gt, -1.f, s.g, s.V));
            RC(vdot(st, s.S[slot], s.Y[slot], s.V, sc(i, S_SY), part));
            RC(vdot(st, s.S[slot], s.S[slot], s.V, sc(i, S_SS), part));
            RC(vdot(st, s.Y[slot], s.Y[slot], s.V, sc(i, S_YY), part));
            if (s.ct) {   // E_c of the accepted point: || c - c_true ||^2 via the scratch vector q
                RC(vaxpby(st, s.q, 1.f, s.xt + s.n0, -1.f, s.ct, nn));
                RC(vdot(st, s.q, s.q, nn, sc(i, S_EC), part));
            }
            if (s.pt) {   // E_p0 over all K data sets: || p0 - p0_true ||^2
                RC(vaxpby(st, s.q, 1.f, s.xt, -1.f, s.pt, s.n0));
                RC(vdot(st, s.q, s.q, s.n0, sc(i, S_EP), part));
            }
        }
        RC(sync_scalars());
        for (int i : act) {
            Inst& s = I[i];
            if (!s.active) continue;
            const int slot = s.next_slot;
            const double sy = hs(i, S_SY), ss = hs(i, S_SS), yy = hs(i, S_YY);
            if (sy > 1e-10 * std::sqrt(ss) * std::sqrt(yy)) {
                const double rho = 1.0 / sy;
                PAT_CUDA(cudaMemcpyAsync(s.rho + slot, &rho, sizeof(double), cudaMemcpyHostToDevice, st));
                RC(set_scalar(i, S_H0, sy / yy));
                s.have_h0 = true;
                if (cfg.mem > 0) {
                    s.order.erase(std::remove(s.order.begin(), s.order.end(), slot), s.order.end());
                    s.order.push_back(slot);
                    if (int(s.order.size()) > cfg.mem) s.order.erase(s.order.begin());
                    s.next_slot = (slot + 1) % memsz;
                } else {
                    s.order.clear();
                }
            }
            const double Jn = hJ[i];
            const double ec = s.ct ? 100.0 * std::sqrt(hs(i, S_EC) / hs(i, S_CT)) : -1.0;
            const double ep = s.pt ? 100.0 * std::sqrt(hs(i, S_EP) / hs(i, S_PT)) : -1.0;
            pat_report* rep = ins[i].report;
            if (rep && rep->count < rep->capacity && rep->iters)
                rep->iters[rep->count++] = pat_iter_report{li,      it, s.J, std::sqrt(hs(i, S_GG)), s.alpha,
                                                           s.trials, Jn, ms_since(s.t_iter), ec, ep};
            const double rel = s.J > 0 ? (s.J - Jn) / s.J : 0.0;
            std::swap(s.z, s.zt);
            std::swap(s.x, s.xt);
            std::swap(s.g, s.gt);
            std::swap(s.zp, s.zpt);
            s.J = Jn;
            if (rel < cfg.rtol) s.active = false;
            // a tracked instance leaves a level (the last one: stops) once every target it
            // has (E_c, E_p0) is reached
            const bool want_c = s.ct && ins[i].ec_target > 0, want_p = s.pt && ins[i].ep0_target > 0;
            if ((want_c || want_p) && (!want_c || ec <= ins[i].ec_target) && (!want_p || ep <= ins[i].ep0_target))
                s.active = false;
        }
    }
    return PAT_OK;
}

int Batch::run() {
    t0 = Clock::now();
    const int Nf = cfg.levels[cfg.nlevels - 1];
    const size_t nnf = size_t(Nf) * Nf;
    hsc.assign(size_t(ni) * S_COUNT, 0.0);
    hJ.assign(ni, 0.0);
    RC(alloc(&dsc, hsc.size()));
    RC(alloc(&part, kPartials));
    RC(alloc(&dJ, ni));
    for (int i = 0; i < ni; ++i)
        if (ins[i].report) {
            ins[i].report->count = 0;
            ins[i].report->status = PAT_OK;
            ins[i].report->total_ms = 0;
        }
    // initial guesses on the finest grid, stacked [K+1][Nf][Nf] per instance
    std::vector<const float*> xprev(ni);
    for (int i = 0; i < ni; ++i) {
        float* xf = nullptr;
        RC(alloc(&xf, size_t(ins[i].K + 1) * nnf));
        PAT_CUDA(cudaMemcpyAsync(xf, ins[i].d_p0_io, ins[i].K * nnf * sizeof(float), cudaMemcpyDeviceToDevice, st));
        PAT_CUDA(cudaMemcpyAsync(xf + ins[i].K * nnf, ins[i].d_c_io, nnf * sizeof(float), cudaMemcpyDeviceToDevice,
                                 st));
        xprev[i] = xf;
    }
    int nprev = Nf;
    int rc = PAT_OK;
    for (int li = 0; li < cfg.nlevels && rc == PAT_OK; ++li) {
        char nvname[64];
        std::snprintf(nvname, sizeof(nvname), "pat_reconstruct level %d (n = %d)", li, cfg.levels[li]);
        NvtxRange nv(nvname);
        rc = level(li, xprev.data(), nprev);
        if (rc != PAT_OK) break;
        for (int i = 0; i < ni; ++i) xprev[i] = I[i].x;
        nprev = N;
    }
    if (rc == PAT_OK) {
        for (int i = 0; i < ni; ++i) {
            PAT_CUDA(cudaMemcpyAsync(ins[i].d_p0_io, xprev[i], ins[i].K * nnf * sizeof(float),
                                     cudaMemcpyDeviceToDevice, st));
            PAT_CUDA(cudaMemcpyAsync(ins[i].d_c_io, xprev[i] + ins[i].K * nnf, nnf * sizeof(float),
                                     cudaMemcpyDeviceToDevice, st));
        }
        PAT_CUDA(cudaStreamSynchronize(st));
        const double tot = ms_since(t0);
        for (int i = 0; i < ni; ++i)
            if (ins[i].report) ins[i].report->total_ms = tot;
    }
    if (plan) pat_plan_destroy(plan);
    plan = nullptr;
    return rc;
}

int check_cfg(const pat_recon_cfg* cfg) {
    if (!cfg || cfg->nlevels < 1 || !cfg->levels || cfg->m < 1 || !cfg->h_sensor_xy || cfg->nt_data < 1 ||
        !(cfg->dt_data > 0) || !(cfg->L > 0) || !(cfg->cfl > 0) || !(cfg->c_hi > cfg->c_lo) || cfg->mem < 0 ||
        cfg->iters < 0 || cfg->max_halvings < 0 || cfg->ckpt_every < 1 || !(cfg->sigma_p0 > 0) ||
        !(cfg->alpha0 > 0) || cfg->prior_tau < 0 ||
        (cfg->prior_tau > 0 && !(cfg->prior_sigma_c > 0 && cfg->prior_sigma_p0 > 0))) {
        set_error("pat_reconstruct: invalid configuration");
        return PAT_EINVAL;
    }
    for (int i = 0; i < cfg->nlevels; ++i)
        if (cfg->levels[i] < 2) { set_error("pat_reconstruct: level side < 2"); return PAT_EINVAL; }
    return PAT_OK;
}

}  // namespace

extern "C" int pat_reconstruct_batched(const pat_recon_cfg* cfg, int ninst, const pat_instance* inst,
                                       void* stream) {
    RC(check_cfg(cfg));
    if (ninst < 1 || !inst) { set_error("pat_reconstruct_batched: need ninst >= 1 instances"); return PAT_EINVAL; }
    for (int i = 0; i < ninst; ++i)
        if (inst[i].K < 1 || !inst[i].d_y_meas || !inst[i].d_w || !inst[i].d_c_io || !inst[i].d_p0_io) {
            set_error("pat_reconstruct_batched: instance %d has a null buffer or K < 1", i);
            return PAT_EINVAL;
        }
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    int rc;
    {
        Batch b(*cfg, ninst, inst, st);
        rc = b.run();
    }
    cudaError_t e = cudaStreamSynchronize(st);
    if (rc == PAT_OK && e != cudaSuccess) rc = cuda_fail(e, "pat_reconstruct");
    return rc;
}

extern "C" int pat_reconstruct(const pat_recon_cfg* cfg, const float* y_meas, const float* w, float* c_io,
                               float* p0_io, pat_report* rep, void* stream) {
    if (!cfg || !y_meas || !w || !c_io || !p0_io) { set_error("pat_reconstruct: null argument"); return PAT_EINVAL; }
    if (cfg->K < 1) { set_error("pat_reconstruct: K < 1"); return PAT_EINVAL; }
    pat_instance one{y_meas, w, c_io, p0_io, cfg->K, rep, nullptr, 0.0, nullptr, 0.0};
    return pat_reconstruct_batched(cfg, 1, &one, stream);
}

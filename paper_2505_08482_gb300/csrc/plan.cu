// Plan creation: grid rules, FP64 tables (wavenumbers, kappa, staggering
// factors, PML profiles, FFT twiddles), bilinear sensor stencils and the
// workspace layout.
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <algorithm>
#include <vector>

#include "pat_internal.h"
#include "kfixed.cuh"
#include "kcluster.cuh"

namespace pat {

static thread_local char g_err[512] = "";

void set_error(const char* fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof(g_err), fmt, ap);
    va_end(ap);
}

int cuda_fail(cudaError_t e, const char* where) {
    set_error("CUDA error %s (%s) in %s", cudaGetErrorName(e), cudaGetErrorString(e), where);
    return PAT_ECUDA;
}

static bool smooth235(int n) {
    if (n < 1) return false;
    for (int q : {2, 3, 5})
        while (n % q == 0) n /= q;
    return n == 1;
}

static bool grid_ok(int ng) { return ng >= 4 && ng <= 1024 && ng % 2 == 0 && smooth235(ng); }

// Radix schedule: as many radix-4 stages as possible, then 5, 3, 2.
bool radix_schedule(int n, FftDesc* fd) {
    fd->n = n;
    fd->nrad = 0;
    int r = n;
    while (r % 4 == 0 && r > 4) {
        fd->rad[fd->nrad++] = 4;
        r /= 4;
    }
    for (int q : {5, 4, 3, 2}) {
        while (r % q == 0) {
            if (fd->nrad >= kMaxStages) return false;
            fd->rad[fd->nrad++] = q;
            r /= q;
        }
    }
    return r == 1;
}

static size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

// PML factor exp(-alpha dt/2) with alpha = pml_alpha (c_ref/dx) (depth/P)^4 at position s (cells).
static double pml_factor(const pat_grid& g, int P, double s) {
    if (P == 0 || g.pml_alpha == 0.0) return 1.0;
    double lo = P - s;
    double hi = s - (P + g.n - 1);
    double xi = std::max(0.0, std::max(lo, hi));
    double q = xi / P;
    double alpha = g.pml_alpha * (g.c_ref / g.dx) * q * q * q * q;
    return std::exp(-0.5 * alpha * g.dt);
}

Ws resolve(const pat_plan_s* p, void* base, bool grad) {
    char* b = static_cast<char*>(base);
    Ws w{};
    const size_t f = size_t(p->K) * p->ng * p->ng;
    float* st = reinterpret_cast<float*>(b + p->o_state);
    w.ux = st;
    w.uy = st + f;
    w.rx = st + 2 * f;
    w.ry = st + 3 * f;
    w.cg = reinterpret_cast<float*>(b + p->o_cg);
    w.A = reinterpret_cast<float2*>(b + p->o_A);
    w.B = reinterpret_cast<float2*>(b + p->o_B);
    w.J = reinterpret_cast<double*>(b + p->o_J);
    w.part = reinterpret_cast<double*>(b + p->o_part);
    w.flag = reinterpret_cast<int*>(b + p->o_flag);
    w.queue = reinterpret_cast<int*>(b + p->o_queue);
    if (grad) {
        w.ckpt = reinterpret_cast<float*>(b + p->o_ckpt);
        w.hist = reinterpret_cast<float*>(b + p->o_hist);
        float* ad = reinterpret_cast<float*>(b + p->o_adj);
        w.ubx = ad;
        w.uby = ad + f;
        w.rbx = ad + 2 * f;
        w.rby = ad + 3 * f;
        w.A2 = reinterpret_cast<float2*>(b + p->o_A2);
        w.B2 = reinterpret_cast<float2*>(b + p->o_B2);
        w.cbar = reinterpret_cast<float*>(b + p->o_cbar);
        w.resid = reinterpret_cast<float*>(b + p->o_resid);
        w.ypred = reinterpret_cast<float*>(b + p->o_ypred);
    }
    return w;
}

static void layout(pat_plan_s* p) {
    const size_t f = size_t(p->K) * p->ng * p->ng * sizeof(float);
    const size_t spec = size_t(p->K) * p->ng * p->hp * sizeof(float2);
    size_t o = 0;
    p->o_state = o; o = align256(o + 4 * f);
    p->o_cg = o; o = align256(o + size_t(p->ninst) * p->ng * p->ng * sizeof(float));
    p->o_A = o; o = align256(o + spec);
    p->o_B = o; o = align256(o + spec);
    p->o_J = o; o = align256(o + size_t(p->ninst) * sizeof(double));
    p->o_part = o; o = align256(o + size_t(p->K) * kResidBlocks * sizeof(double));
    p->o_flag = o; o = align256(o + 4 * sizeof(int));
    p->o_queue = o; o = align256(o + (size_t(p->K) + 2) * sizeof(int));
    p->ws_fwd = o;
    p->o_ckpt = o; o = align256(o + size_t(std::max(p->nseg - 1, 0)) * 4 * f);
    p->o_hist = o; o = align256(o + size_t(p->nseg > 1 ? 2 : 1) * p->K * p->s_eff * p->ng * p->ng * sizeof(float));
    p->o_adj = o; o = align256(o + 4 * f);
    p->o_A2 = o; o = align256(o + spec);
    p->o_B2 = o; o = align256(o + spec);
    p->o_cbar = o; o = align256(o + size_t(p->K) * p->n * p->n * sizeof(float));
    const size_t tr = size_t(p->K) * p->nt * p->m * sizeof(float);
    p->o_resid = o; o = align256(o + tr);
    p->o_ypred = o; o = align256(o + tr);
    p->ws_grad = o;
}

}  // namespace pat

using namespace pat;

extern "C" const char* pat_last_error(void) { return g_err; }

extern "C" int pat_pml_auto(int n, int min_pml) {
    if (n < 2 || min_pml < 0) return -1;
    for (int P = min_pml; n + 2 * P <= 1024; ++P)
        if (grid_ok(n + 2 * P)) return P;
    return -1;
}

extern "C" int pat_plan_ng(pat_plan plan) { return plan ? plan->ng : -1; }

extern "C" int pat_plan_shape(pat_plan plan, int* ninst, int* K) {
    if (!plan || !ninst || !K) { set_error("pat_plan_shape: null argument"); return PAT_EINVAL; }
    *ninst = plan->ninst;
    *K = plan->K;
    return PAT_OK;
}

extern "C" int pat_plan_variants(pat_plan plan) { return plan ? fixed_variants(plan->ng) : -1; }

extern "C" int pat_plan_set_variant(pat_plan plan, int variant) {
    if (!plan) { set_error("pat_plan_set_variant: null plan"); return PAT_EINVAL; }
    if (variant >= fixed_variants(plan->ng)) {
        set_error("pat_plan_set_variant: grid side %d has %d fixed-size variants", plan->ng, fixed_variants(plan->ng));
        return PAT_EINVAL;
    }
    return select_variant(plan, variant < 0 ? -1 : variant);
}

extern "C" int pat_plan_variant(pat_plan plan) { return plan ? plan->variant : -2; }

extern "C" int pat_plan_set_persistent(pat_plan plan, int enable) {
    if (!plan) { set_error("pat_plan_set_persistent: null plan"); return PAT_EINVAL; }
    if (!enable) {
        plan->persistent = false;
        return PAT_OK;
    }
    const SweepOps* so = sweep_ops_for(plan->ng);
    if (!so) {
        set_error("pat_plan_set_persistent: grid side %d has no persistent sweep (sides 108, 144, 180, 200, 240, 300)",
                  plan->ng);
        return PAT_EINVAL;
    }
    int rc = so->configure();
    if (rc != PAT_OK) return rc;
    plan->sweep = so;
    plan->persistent = true;
    return PAT_OK;
}

extern "C" int pat_plan_persistent(pat_plan plan) { return plan ? int(plan->persistent) : -1; }

extern "C" int pat_plan_set_cluster(pat_plan plan, int enable) {
    if (!plan) { set_error("pat_plan_set_cluster: null plan"); return PAT_EINVAL; }
    if (!enable) {
        plan->cluster = false;
        return PAT_OK;
    }
    const ClusterOps* co = cluster_ops_for(plan->ng);
    if (!co) {
        set_error("pat_plan_set_cluster: grid side %d has no cluster-resident stepping (side 300)", plan->ng);
        return PAT_EINVAL;
    }
    int rc = co->configure();
    if (rc != PAT_OK) return rc;
    plan->clops = co;
    plan->cluster = true;
    return PAT_OK;
}

extern "C" int pat_plan_cluster(pat_plan plan) { return plan ? int(plan->cluster) : -1; }

extern "C" int pat_plan_cluster_capacity(pat_plan plan) {
    if (!plan) { set_error("pat_plan_cluster_capacity: null plan"); return PAT_EINVAL; }
    const ClusterOps* co = plan->clops ? plan->clops : cluster_ops_for(plan->ng);
    if (!co || co->configure() != PAT_OK) return 0;
    return co->capacity();
}

extern "C" int pat_plan_set_graphs(pat_plan plan, int enable) {
    if (!plan) { set_error("pat_plan_set_graphs: null plan"); return PAT_EINVAL; }
    plan->use_graphs = enable != 0;
    if (!plan->use_graphs) {
        for (auto& g : plan->graphs) cudaGraphExecDestroy(g.exec);
        plan->graphs.clear();
    }
    return PAT_OK;
}

extern "C" int pat_plan_create(pat_plan* out, const pat_grid* g, int m, const double* xy, int K,
                               int ckpt_every) {
    return pat_plan_create_batched(out, g, m, xy, 1, &K, ckpt_every);
}

extern "C" int pat_plan_create_batched(pat_plan* out, const pat_grid* g, int m, const double* xy, int ninst,
                                       const int* h_K, int ckpt_every) {
    if (!out || !g || !h_K) { set_error("pat_plan_create: null argument"); return PAT_EINVAL; }
    *out = nullptr;
    if (ninst < 1 || ninst > 65536) { set_error("pat_plan_create: need 1 <= ninst <= 65536"); return PAT_EINVAL; }
    long long Ktot = 0;
    for (int i = 0; i < ninst; ++i) {
        if (h_K[i] < 1) { set_error("pat_plan_create: instance %d has K < 1", i); return PAT_EINVAL; }
        Ktot += h_K[i];
    }
    if (Ktot > 65535) { set_error("pat_plan_create: at most 65535 data sets per plan"); return PAT_EINVAL; }
    const int K = int(Ktot);
    if (g->n < 2 || g->pml < 0 || g->nt < 1 || m < 1 || !xy || ckpt_every < 1) {
        set_error("pat_plan_create: need n>=2, pml>=0, nt>=1, K>=1, m>=1, sensors, ckpt_every>=1");
        return PAT_EINVAL;
    }
    if (!(g->dx > 0) || !(g->dt > 0) || !(g->c_ref > 0) || !(g->rho0 > 0) || !(g->c_bg > 0) ||
        !(g->pml_alpha >= 0)) {
        set_error("pat_plan_create: dx, dt, c_ref, rho0, c_bg must be > 0 and pml_alpha >= 0");
        return PAT_EINVAL;
    }
    const int ng = g->n + 2 * g->pml;
    if (!grid_ok(ng)) {
        set_error("pat_plan_create: grid side n+2*pml = %d must be even, 5-smooth and <= 1024", ng);
        return PAT_EINVAL;
    }
    pat_plan_s* p = new pat_plan_s();
    p->g = *g;
    p->n = g->n;
    p->P = g->pml;
    p->ng = ng;
    p->hc = ng / 2 + 1;
    p->hp = (p->hc + 3) & ~3;
    p->K = K;
    p->ninst = ninst;
    p->nt = g->nt;
    p->m = m;
    p->s = ckpt_every;
    p->s_eff = std::min(ckpt_every, g->nt);
    p->nseg = (g->nt + p->s_eff - 1) / p->s_eff;
    p->hist_valid_ws = nullptr;
    p->sweep = nullptr;
    p->persistent = false;
    p->clops = nullptr;
    p->cluster = false;
    p->use_graphs = false;
    p->graph_clock = 0;
    p->side = nullptr;
    p->ev_start = p->ev_rec[0] = p->ev_rec[1] = p->ev_adj[0] = p->ev_adj[1] = nullptr;
    cudaGetDevice(&p->device);
    radix_schedule(ng, &p->fft);

    // ---- FP64 tables ----
    const double dx = g->dx, dt = g->dt;
    const double PI = 3.14159265358979323846;
    std::vector<double> k1(ng);
    for (int i = 0; i < ng; ++i) {
        int q = (i < ng / 2) ? i : i - ng;     // {0..ng/2-1, -ng/2..-1}
        k1[i] = 2.0 * PI * q / (ng * dx);
    }
    std::vector<float2> tw(ng), fx(p->hc), fy(ng);
    for (int q = 0; q < ng; ++q) {
        double a = -2.0 * PI * q / ng;
        tw[q] = make_float2(float(std::cos(a)), float(std::sin(a)));
    }
    auto gfac = [&](double k, bool nyq) {
        // i k exp(+i k dx/2); real at the Nyquist wavenumber
        double c = std::cos(0.5 * k * dx), s = std::sin(0.5 * k * dx);
        double re = -k * s, im = k * c;
        if (nyq) im = 0.0;
        return make_float2(float(re), float(im));
    };
    for (int i = 0; i < p->hc; ++i) fx[i] = gfac(k1[i], i == ng / 2);
    for (int i = 0; i < ng; ++i) fy[i] = gfac(k1[i], i == ng / 2);
    std::vector<float> kap(size_t(p->hc) * ng);
    for (int kx = 0; kx < p->hc; ++kx)
        for (int ky = 0; ky < ng; ++ky) {
            double kk = std::sqrt(k1[kx] * k1[kx] + k1[ky] * k1[ky]);
            double a = 0.5 * g->c_ref * kk * dt;
            kap[size_t(kx) * ng + ky] = float(a == 0.0 ? 1.0 : std::sin(a) / a);
        }
    std::vector<float> ac(ng), as(ng);
    for (int i = 0; i < ng; ++i) {
        ac[i] = float(pml_factor(*g, p->P, double(i)));
        as[i] = float(pml_factor(*g, p->P, i + 0.5));
    }
    // ---- sensor stencils, CSR by grid row ----
    struct Ent { int row, m, ix; float wx0, wx1, wy; };
    std::vector<Ent> ents;
    ents.reserve(2 * m);
    for (int s = 0; s < m; ++s) {
        double gx = xy[2 * s] / dx - 0.5 + p->P;
        double gy = xy[2 * s + 1] / dx - 0.5 + p->P;
        if (!std::isfinite(gx) || !std::isfinite(gy)) {
            set_error("pat_plan_create: sensor %d has a non-finite position", s);
            delete p;
            return PAT_EINVAL;
        }
        int ix = int(std::floor(gx)), iy = int(std::floor(gy));
        if (ix < 0 || iy < 0 || ix + 1 > ng - 1 || iy + 1 > ng - 1) {
            set_error("pat_plan_create: sensor %d at (%g, %g) m lies outside the grid", s, xy[2 * s], xy[2 * s + 1]);
            delete p;
            return PAT_EINVAL;
        }
        double fxr = gx - ix, fyr = gy - iy;
        ents.push_back({iy, s, ix, float(1.0 - fxr), float(fxr), float(1.0 - fyr)});
        ents.push_back({iy + 1, s, ix, float(1.0 - fxr), float(fxr), float(fyr)});
    }
    std::stable_sort(ents.begin(), ents.end(), [](const Ent& a, const Ent& b) { return a.row < b.row; });
    p->nent = int(ents.size());
    std::vector<int> srow(ng + 1, 0);
    for (const Ent& e : ents) srow[e.row + 1]++;
    for (int i = 0; i < ng; ++i) srow[i + 1] += srow[i];
    std::vector<int> kinst(K), kfirst(ninst + 1, 0);
    for (int i = 0, k = 0; i < ninst; ++i) {
        kfirst[i] = k;
        for (int j = 0; j < h_K[i]; ++j) kinst[k++] = i;
    }
    kfirst[ninst] = K;
    std::vector<int2> sent(p->nent);
    std::vector<float4> sentw(p->nent);
    for (int i = 0; i < p->nent; ++i) {
        sent[i] = make_int2(ents[i].m, ents[i].ix);
        sentw[i] = make_float4(ents[i].wx0, ents[i].wx1, ents[i].wy, float(ents[i].row));
    }

    // ---- one device allocation for all tables ----
    size_t o = 0;
    auto take = [&](size_t bytes) { size_t r = o; o = align256(o + bytes); return r; };
    size_t o_tw = take(ng * sizeof(float2)), o_k = take(kap.size() * sizeof(float));
    size_t o_fx = take(p->hc * sizeof(float2)), o_fy = take(ng * sizeof(float2));
    size_t o_ac = take(ng * sizeof(float)), o_as = take(ng * sizeof(float));
    size_t o_sr = take((ng + 1) * sizeof(int)), o_se = take(p->nent * sizeof(int2));
    size_t o_sw = take(p->nent * sizeof(float4));
    size_t o_ki = take(K * sizeof(int)), o_kf = take((ninst + 1) * sizeof(int));
    cudaError_t e = cudaMalloc(&p->dev, o);
    if (e != cudaSuccess) {
        cuda_fail(e, "cudaMalloc(plan tables)");
        delete p;
        return PAT_ENOMEM;
    }
    char* d = static_cast<char*>(p->dev);
    p->t.tw = reinterpret_cast<float2*>(d + o_tw);
    p->t.kappa_t = reinterpret_cast<float*>(d + o_k);
    p->t.fx = reinterpret_cast<float2*>(d + o_fx);
    p->t.fy = reinterpret_cast<float2*>(d + o_fy);
    p->t.a_cell = reinterpret_cast<float*>(d + o_ac);
    p->t.a_stag = reinterpret_cast<float*>(d + o_as);
    p->t.srow = reinterpret_cast<int*>(d + o_sr);
    p->t.sent = reinterpret_cast<int2*>(d + o_se);
    p->t.sentw = reinterpret_cast<float4*>(d + o_sw);
    p->t.kinst = reinterpret_cast<int*>(d + o_ki);
    p->t.kfirst = reinterpret_cast<int*>(d + o_kf);
    struct Cp { void* dst; const void* src; size_t n; } cps[] = {
        {p->t.tw, tw.data(), ng * sizeof(float2)},
        {p->t.kappa_t, kap.data(), kap.size() * sizeof(float)},
        {p->t.fx, fx.data(), p->hc * sizeof(float2)},
        {p->t.fy, fy.data(), ng * sizeof(float2)},
        {p->t.a_cell, ac.data(), ng * sizeof(float)},
        {p->t.a_stag, as.data(), ng * sizeof(float)},
        {p->t.srow, srow.data(), (ng + 1) * sizeof(int)},
        {p->t.sent, sent.data(), p->nent * sizeof(int2)},
        {p->t.sentw, sentw.data(), p->nent * sizeof(float4)},
        {p->t.kinst, kinst.data(), K * sizeof(int)},
        {p->t.kfirst, kfirst.data(), (ninst + 1) * sizeof(int)},
    };
    for (const Cp& c : cps)
        if (e == cudaSuccess) e = cudaMemcpy(c.dst, c.src, c.n, cudaMemcpyHostToDevice);
    // copies from pageable memory may still be in flight when cudaMemcpy returns, and the
    // caller's non-blocking streams are not ordered after the legacy stream: wait for them
    if (e == cudaSuccess) e = cudaStreamSynchronize(cudaStreamLegacy);
    if (e != cudaSuccess) {
        int rc = cuda_fail(e, "cudaMemcpy(plan tables)");
        cudaFree(p->dev);
        delete p;
        return rc;
    }
    p->R = 8;
    p->C = 4;
    int rc = configure_kernels(p);
    if (rc != PAT_OK) {
        cudaFree(p->dev);
        delete p;
        return rc;
    }
    layout(p);
    if (cudaStreamCreateWithFlags(&p->side, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&p->ev_start, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&p->ev_rec[0], cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&p->ev_rec[1], cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&p->ev_adj[0], cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&p->ev_adj[1], cudaEventDisableTiming) != cudaSuccess) {
        int rc2 = cuda_fail(cudaGetLastError(), "pat_plan_create (stream, events)");
        pat_plan_destroy(p);
        return rc2;
    }
    *out = p;
    return PAT_OK;
}

extern "C" void pat_plan_destroy(pat_plan p) {
    if (!p) return;
    for (auto& g : p->graphs) cudaGraphExecDestroy(g.exec);
    for (cudaEvent_t e : {p->ev_start, p->ev_rec[0], p->ev_rec[1], p->ev_adj[0], p->ev_adj[1]})
        if (e) cudaEventDestroy(e);
    if (p->side) {
        cudaStreamSynchronize(p->side);
        cudaStreamDestroy(p->side);
    }
    if (p->dev) cudaFree(p->dev);
    delete p;
}

extern "C" size_t pat_workspace_bytes(pat_plan p, int kind) {
    if (!p) return 0;
    return kind == PAT_WS_GRADIENT ? p->ws_grad : p->ws_fwd;
}

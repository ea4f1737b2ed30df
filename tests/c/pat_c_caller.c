/*
 * A plain C caller of libpat (no Python, no C++): the forward traces and the
 * gradient of the data term for inputs read from raw files, results written
 * back as raw files.  tests/test_gpu_c_caller.py compiles it with gcc against
 * include/pat.h and the CUDA runtime, runs it and compares its outputs with
 * the Python binding's on the same inputs; tests/test_c_caller_host.py only
 * compiles and links it.
 *
 * Usage: pat_c_caller DIR.  DIR/meta.txt holds "n pml dx dt nt c_ref rho0
 * pml_alpha c_bg m K ckpt_every"; DIR/{c,p0,y_meas,w}.f32 and DIR/xy.f64 are
 * the inputs (c [n][n], p0 [K][n][n], y_meas [K][nt][m], w [K] float32;
 * sensor positions [m][2] float64 in metres).  Writes DIR/{y,grad_p0,grad_c}.f32
 * and DIR/J.f64.  Exit status 0 on success, 1 on a library or CUDA error
 * (message on stderr).
 */
#include <stdio.h>
#include <stdlib.h>

#include <cuda_runtime_api.h>

#include "pat.h"

static void* read_raw(const char* dir, const char* name, size_t bytes) {
    char path[4096];
    snprintf(path, sizeof(path), "%s/%s", dir, name);
    FILE* f = fopen(path, "rb");
    if (!f) return NULL;
    void* buf = malloc(bytes);
    size_t got = buf ? fread(buf, 1, bytes, f) : 0;
    fclose(f);
    if (got != bytes) {
        free(buf);
        return NULL;
    }
    return buf;
}

static int write_raw(const char* dir, const char* name, const void* buf, size_t bytes) {
    char path[4096];
    snprintf(path, sizeof(path), "%s/%s", dir, name);
    FILE* f = fopen(path, "wb");
    if (!f) return 1;
    size_t put = fwrite(buf, 1, bytes, f);
    fclose(f);
    return put == bytes ? 0 : 1;
}

#define CK(call)                                                             \
    do {                                                                     \
        cudaError_t e_ = (call);                                             \
        if (e_ != cudaSuccess) {                                             \
            fprintf(stderr, "%s: %s\n", #call, cudaGetErrorString(e_));     \
            return 1;                                                        \
        }                                                                    \
    } while (0)

#define PK(call)                                                             \
    do {                                                                     \
        int rc_ = (call);                                                    \
        if (rc_ != PAT_OK) {                                                 \
            fprintf(stderr, "%s: %d %s\n", #call, rc_, pat_last_error());   \
            return 1;                                                        \
        }                                                                    \
    } while (0)

int main(int argc, char** argv) {
    if (argc != 2) {
        fprintf(stderr, "usage: %s DIR\n", argv[0]);
        return 1;
    }
    const char* dir = argv[1];
    char path[4096];
    snprintf(path, sizeof(path), "%s/meta.txt", dir);
    FILE* mf = fopen(path, "r");
    if (!mf) {
        fprintf(stderr, "cannot open %s\n", path);
        return 1;
    }
    pat_grid g;
    int m = 0, K = 0, ckpt = 0;
    int got = fscanf(mf, "%d %d %lf %lf %d %lf %lf %lf %lf %d %d %d", &g.n, &g.pml, &g.dx, &g.dt, &g.nt, &g.c_ref,
                     &g.rho0, &g.pml_alpha, &g.c_bg, &m, &K, &ckpt);
    fclose(mf);
    if (got != 12 || g.n < 1 || m < 1 || K < 1 || g.nt < 1) {
        fprintf(stderr, "bad meta.txt\n");
        return 1;
    }
    const size_t nn = (size_t)g.n * g.n, ny = (size_t)K * g.nt * m;
    float* c = read_raw(dir, "c.f32", nn * sizeof(float));
    float* p0 = read_raw(dir, "p0.f32", K * nn * sizeof(float));
    float* ym = read_raw(dir, "y_meas.f32", ny * sizeof(float));
    float* w = read_raw(dir, "w.f32", K * sizeof(float));
    double* xy = read_raw(dir, "xy.f64", 2 * (size_t)m * sizeof(double));
    if (!c || !p0 || !ym || !w || !xy) {
        fprintf(stderr, "missing or short input file\n");
        return 1;
    }

    pat_plan plan = NULL;
    PK(pat_plan_create(&plan, &g, m, xy, K, ckpt));
    const size_t wsb = pat_workspace_bytes(plan, PAT_WS_GRADIENT);
    void *d_ws = NULL, *d_c = NULL, *d_p0 = NULL, *d_y = NULL, *d_ym = NULL, *d_w = NULL, *d_gp0 = NULL,
         *d_gc = NULL, *d_J = NULL;
    CK(cudaMalloc(&d_ws, wsb));
    CK(cudaMalloc(&d_c, nn * sizeof(float)));
    CK(cudaMalloc(&d_p0, K * nn * sizeof(float)));
    CK(cudaMalloc(&d_y, ny * sizeof(float)));
    CK(cudaMalloc(&d_ym, ny * sizeof(float)));
    CK(cudaMalloc(&d_w, K * sizeof(float)));
    CK(cudaMalloc(&d_gp0, K * nn * sizeof(float)));
    CK(cudaMalloc(&d_gc, nn * sizeof(float)));
    CK(cudaMalloc(&d_J, sizeof(double)));
    CK(cudaMemcpy(d_c, c, nn * sizeof(float), cudaMemcpyHostToDevice));
    CK(cudaMemcpy(d_p0, p0, K * nn * sizeof(float), cudaMemcpyHostToDevice));
    CK(cudaMemcpy(d_ym, ym, ny * sizeof(float), cudaMemcpyHostToDevice));
    CK(cudaMemcpy(d_w, w, K * sizeof(float), cudaMemcpyHostToDevice));

    PK(pat_forward(plan, d_c, d_p0, d_y, d_ws, wsb, NULL));
    PK(pat_adjoint_grad(plan, d_c, d_p0, d_ym, d_w, d_gp0, d_gc, d_J, NULL, d_ws, wsb, NULL));
    CK(cudaDeviceSynchronize());
    int flag = 0;
    PK(pat_status(plan, d_ws, &flag, NULL));

    float* y = malloc(ny * sizeof(float));
    float* gp0 = malloc(K * nn * sizeof(float));
    float* gc = malloc(nn * sizeof(float));
    double J = 0.0;
    if (!y || !gp0 || !gc) return 1;
    CK(cudaMemcpy(y, d_y, ny * sizeof(float), cudaMemcpyDeviceToHost));
    CK(cudaMemcpy(gp0, d_gp0, K * nn * sizeof(float), cudaMemcpyDeviceToHost));
    CK(cudaMemcpy(gc, d_gc, nn * sizeof(float), cudaMemcpyDeviceToHost));
    CK(cudaMemcpy(&J, d_J, sizeof(double), cudaMemcpyDeviceToHost));
    if (write_raw(dir, "y.f32", y, ny * sizeof(float)) || write_raw(dir, "grad_p0.f32", gp0, K * nn * sizeof(float)) ||
        write_raw(dir, "grad_c.f32", gc, nn * sizeof(float)) || write_raw(dir, "J.f64", &J, sizeof(double))) {
        fprintf(stderr, "cannot write the outputs\n");
        return 1;
    }
    printf("J %.17g status %d\n", J, flag);

    pat_plan_destroy(plan);
    void* bufs[] = {d_ws, d_c, d_p0, d_y, d_ym, d_w, d_gp0, d_gc, d_J};
    for (size_t i = 0; i < sizeof(bufs) / sizeof(bufs[0]); ++i) cudaFree(bufs[i]);
    free(c);
    free(p0);
    free(ym);
    free(w);
    free(xy);
    free(y);
    free(gp0);
    free(gc);
    return 0;
}

// qsmg_host.cu -- host side of the C ABI declared in include/qsmg.h:
// hierarchy set-up (Galerkin coarse operators, dense coarsest inverse),
// V-cycle and solve orchestration (FP64, and FP32 cycles inside FP64
// iterative refinement), the projection step, and the component entry points.
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <vector>

#include "../../include/qsmg.h"
#include "qsmg_impl.h"

using namespace qsmg;

namespace {

thread_local char g_err[512] = "";

void set_err(const char *fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof(g_err), fmt, ap);
    va_end(ap);
}

constexpr int kMaxLev = 16;
constexpr int kMaxCoarse = 3072;
constexpr int kProfSlots = 64;
constexpr int kMaxInner = 10;  // cap on FP32 V-cycles per refinement step

// n FP32 V-cycles (from e = 0) captured once and replayed; the event pairs
// around its finest-level smoothing calls are recorded by every replay
struct InnerGraph {
    cudaGraphExec_t exec = nullptr;
    long kernels = 0;
    int nev = 0;
    cudaEvent_t ev[2 * kMaxInner][2];
    long sweeps[2 * kMaxInner], launches[2 * kMaxInner];
};

}  // namespace

std::atomic<long> qsmg::g_launches{0};

void qsmg::set_last_error(const char *fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof(g_err), fmt, ap);
    va_end(ap);
}

struct mg_ctx {
    int nlev;
    Dims L[kMaxLev];
    double S[kMaxLev][243];  // host stencil tables of the scaled operator
    Fine<double> f64;
    Fine<float> f32;
    Coarse<double> c64[kMaxLev];
    Coarse<float> c32[kMaxLev];
    double lam, mu, h;
    mg_bc bc;
    stz_params stz;
    bool has_bc, has_stz;
    mg_opts opts;
    cudaStream_t st;
    bool broken;
    // device buffers (level 0 x/b in FP64 mode are the caller's arrays)
    double *x64[kMaxLev], *b64[kMaxLev], *r64[kMaxLev];
    float *x32[kMaxLev], *b32[kMaxLev], *r32[kMaxLev];
    float *xs32[kMaxLev];  // ping-pong partners of the tiled FP32 sweeps
    int split0;            // finest FP32 arrays in parity-split column order
    double *Ainv;
    int ncoarse;
    double *partials, *dsum, *hsum;
    // cross-CTA state of the fused finest-level sweep (when it applies)
    SweepSync sync;
    bool has_sync;
    int *herr;  // pinned host copy of its error word
    double *sig_star, *dpl, *sbar, *chi_tmp, *rhs;
    // adjoint-step scratch, allocated at the first qs_step_adjoint
    double *adj_rhs, *adj_lam, *adj_cb, *adj_db, *adj_sbb, *adj_sgb, *adj_Lb;
    // finest-level smoothing timers (event pairs recorded on st)
    bool prof_on, prof_events;
    cudaEvent_t ev[kProfSlots][2];
    cudaEvent_t pend_ev[kProfSlots][2];
    long pend_sweeps[kProfSlots], pend_launches[kProfSlots];
    int npend;
    // FP32 inner V-cycles as CUDA graphs, one per cycle count
    InnerGraph *graphs[kMaxInner + 1];
    cudaStream_t cap;  // private stream used only to capture them
    InnerGraph *capturing;
    double prof_ms;
    long prof_sweeps, prof_launches;
    std::vector<void *> allocs;
};

#define CK(expr)                                                                        \
    do {                                                                                \
        cudaError_t e_ = (expr);                                                        \
        if (e_ != cudaSuccess) {                                                        \
            set_err("%s failed: %s (%s:%d)", #expr, cudaGetErrorString(e_), __FILE__, \
                    __LINE__);                                                          \
            if (ctx) ctx->broken = true;                                                \
            return MG_ERR_CUDA;                                                         \
        }                                                                               \
    } while (0)

#define CKS(expr)                         \
    do {                                  \
        mg_status s_ = (expr);            \
        if (s_ != MG_OK) return s_;       \
    } while (0)

namespace {

// ---------------------------------------------------------------- set-up

// Scaled finest-level stencil (27, 3, 3): Eq. (30) with the collocated
// 3-point second derivative (Eq. 32) and 4-point mixed derivative of
// section 3.4, multiplied by -h^2/(mu dt).
void fine_table(double lam, double mu, double *S) {
    const double lp = (lam + 2.0 * mu) / mu, kq = (lam + mu) / (4.0 * mu);
    memset(S, 0, 243 * sizeof(double));
    auto at = [&](int dx, int dy, int dz, int a, int b) -> double & {
        return S[((dz + 1) * 9 + (dy + 1) * 3 + (dx + 1)) * 9 + a * 3 + b];
    };
    for (int a = 0; a < 3; a++) at(0, 0, 0, a, a) = 2.0 * lp + 4.0;
    for (int ax = 0; ax < 3; ax++)
        for (int s = -1; s <= 1; s += 2) {
            int o[3] = {0, 0, 0};
            o[ax] = s;
            for (int a = 0; a < 3; a++) at(o[0], o[1], o[2], a, a) = (a == ax) ? -lp : -1.0;
        }
    for (int a = 0; a < 3; a++)
        for (int b = 0; b < 3; b++) {
            if (a == b) continue;
            for (int sa = -1; sa <= 1; sa += 2)
                for (int sb = -1; sb <= 1; sb += 2) {
                    int o[3] = {0, 0, 0};
                    o[a] = sa;
                    o[b] = sb;
                    at(o[0], o[1], o[2], a, b) = -kq * sa * sb;
                }
        }
}

// Galerkin coarse stencil A_c = R A T (Eq. 36) in two separable stages:
//   AT(g)  = sum_f t(f) A(g + f)          g in [-3, 3]^3  (operator times interpolation)
//   A_c(D) = sum_e t(e) AT(2D - e)        D in [-1, 1]^3  (restriction, stride 2)
// with the trilinear weights t(e) = prod (1 - |e_axis|/2).
void galerkin_table(const double *Sf, double *Sc) {
    static double AT[7][7][7][9];
    memset(AT, 0, sizeof(AT));
    auto t1 = [](int e) { return e == 0 ? 1.0 : 0.5; };
    for (int gz = -3; gz <= 3; gz++)
        for (int gy = -3; gy <= 3; gy++)
            for (int gx = -3; gx <= 3; gx++)
                for (int fz = -1; fz <= 1; fz++)
                    for (int fy = -1; fy <= 1; fy++)
                        for (int fx = -1; fx <= 1; fx++) {
                            const int ax = gx + fx, ay = gy + fy, az = gz + fz;
                            if (ax < -1 || ax > 1 || ay < -1 || ay > 1 || az < -1 || az > 1)
                                continue;
                            const double w = t1(fx) * t1(fy) * t1(fz);
                            const double *a = Sf + ((az + 1) * 9 + (ay + 1) * 3 + (ax + 1)) * 9;
                            double *o = AT[gz + 3][gy + 3][gx + 3];
                            for (int m = 0; m < 9; m++) o[m] += w * a[m];
                        }
    memset(Sc, 0, 243 * sizeof(double));
    for (int Dz = -1; Dz <= 1; Dz++)
        for (int Dy = -1; Dy <= 1; Dy++)
            for (int Dx = -1; Dx <= 1; Dx++) {
                double *o = Sc + ((Dz + 1) * 9 + (Dy + 1) * 3 + (Dx + 1)) * 9;
                for (int ez = -1; ez <= 1; ez++)
                    for (int ey = -1; ey <= 1; ey++)
                        for (int ex = -1; ex <= 1; ex++) {
                            const double w = t1(ex) * t1(ey) * t1(ez);
                            const double *a = AT[2 * Dz - ez + 3][2 * Dy - ey + 3][2 * Dx - ex + 3];
                            for (int m = 0; m < 9; m++) o[m] += w * a[m];
                        }
            }
}

// Parity-class form of a 27 x 3 x 3 stencil table (see Coarse<T>): the
// class values are the means of their members; false when an entry departs
// from its class value by more than 1e-12 of the largest entry (a table
// without the reflection symmetry) or a centre entry is not positive
bool parity_classes(const double *S, Coarse<double> &c) {
    double mx = 0.0;
    for (int m = 0; m < 243; m++) mx = fmax(mx, fabs(S[m]));
    double cs[3][8] = {}, gs[3][2] = {};
    int cn[3][8] = {}, gn[3][2] = {};
    auto sgn = [](int v) { return v > 0 ? 1.0 : -1.0; };
    for (int dz = -1; dz <= 1; dz++)
        for (int dy = -1; dy <= 1; dy++)
            for (int dx = -1; dx <= 1; dx++) {
                const int dd = (dz + 1) * 9 + (dy + 1) * 3 + (dx + 1), dv[3] = {dx, dy, dz};
                const int cls = abs(dx) + 2 * abs(dy) + 4 * abs(dz);
                for (int a = 0; a < 3; a++) {
                    cs[a][cls] += S[dd * 9 + 4 * a];
                    cn[a][cls]++;
                    for (int b = 0; b < 3; b++)
                        if (b != a && dv[a] && dv[b]) {
                            const int t = 3 - a - b;
                            gs[t][abs(dv[t])] += sgn(dv[a]) * sgn(dv[b]) * S[dd * 9 + 3 * a + b];
                            gn[t][abs(dv[t])]++;
                        }
                }
            }
    for (int a = 0; a < 3; a++) {
        for (int m = 0; m < 8; m++) c.cd[a][m] = cs[a][m] / cn[a][m];
        for (int m = 0; m < 2; m++) c.g[a][m] = gs[a][m] / gn[a][m];
        if (!(c.cd[a][0] > 0.0)) return false;
        c.dinv[a] = 1.0 / c.cd[a][0];
    }
    // every entry against the value its class gives it
    for (int dz = -1; dz <= 1; dz++)
        for (int dy = -1; dy <= 1; dy++)
            for (int dx = -1; dx <= 1; dx++) {
                const int dd = (dz + 1) * 9 + (dy + 1) * 3 + (dx + 1), dv[3] = {dx, dy, dz};
                const int cls = abs(dx) + 2 * abs(dy) + 4 * abs(dz);
                for (int a = 0; a < 3; a++)
                    for (int b = 0; b < 3; b++) {
                        double want = 0.0;
                        if (a == b)
                            want = c.cd[a][cls];
                        else if (dv[a] && dv[b])
                            want = sgn(dv[a]) * sgn(dv[b]) * c.g[3 - a - b][abs(dv[3 - a - b])];
                        if (fabs(S[dd * 9 + 3 * a + b] - want) > 1e-12 * mx) return false;
                    }
            }
    return true;
}

// dense inverse of the coarsest operator (interior unknowns, ordering
// u = (((k-1) ny + j) nx + i) * 3 + a) via a Cholesky factorisation
bool coarse_inverse(const Dims &d, const double *S, std::vector<double> &Ainv) {
    const int nx = d.nx, ny = d.ny, nz = d.nz;
    const int n = 3 * nx * ny * (nz - 1);
    std::vector<double> A((size_t)n * n, 0.0);
    auto unk = [&](int a, int k, int j, int i) { return (((k - 1) * ny + j) * nx + i) * 3 + a; };
    for (int k = 1; k < nz; k++)
        for (int j = 0; j < ny; j++)
            for (int i = 0; i < nx; i++)
                for (int dd = 0; dd < 27; dd++) {
                    const int dz = dd / 9 - 1, dy = (dd / 3) % 3 - 1, dx = dd % 3 - 1;
                    const int kk = k + dz;
                    if (kk < 1 || kk >= nz) continue;
                    const int jj = (j + dy + ny) % ny, ii = (i + dx + nx) % nx;
                    for (int a = 0; a < 3; a++)
                        for (int b = 0; b < 3; b++)
                            A[(size_t)unk(a, k, j, i) * n + unk(b, kk, jj, ii)] += S[dd * 9 + a * 3 + b];
                }
    // Cholesky A = L L^T (lower part of A overwritten)
    for (int c = 0; c < n; c++) {
        double s = A[(size_t)c * n + c];
        for (int p = 0; p < c; p++) s -= A[(size_t)c * n + p] * A[(size_t)c * n + p];
        if (!(s > 0.0)) return false;
        const double l = sqrt(s);
        A[(size_t)c * n + c] = l;
        for (int r = c + 1; r < n; r++) {
            double t = A[(size_t)r * n + c];
            for (int p = 0; p < c; p++) t -= A[(size_t)r * n + p] * A[(size_t)c * n + p];
            A[(size_t)r * n + c] = t / l;
        }
    }
    Ainv.assign((size_t)n * n, 0.0);
    std::vector<double> y(n);
    for (int col = 0; col < n; col++) {
        for (int r = 0; r < n; r++) {
            double s = (r == col) ? 1.0 : 0.0;
            for (int p = 0; p < r; p++) s -= A[(size_t)r * n + p] * y[p];
            y[r] = s / A[(size_t)r * n + r];
        }
        for (int r = n - 1; r >= 0; r--) {
            double s = y[r];
            for (int p = r + 1; p < n; p++) s -= A[(size_t)p * n + r] * y[p];
            y[r] = s / A[(size_t)r * n + r];
        }
        for (int r = 0; r < n; r++) Ainv[(size_t)r * n + col] = y[r];
    }
    return true;
}

template <typename T>
mg_status dalloc(mg_ctx *ctx, T **p, size_t count) {
    void *q = nullptr;
    cudaError_t e = cudaMalloc(&q, count * sizeof(T));
    if (e != cudaSuccess) {
        set_err("cudaMalloc of %zu bytes failed: %s", count * sizeof(T), cudaGetErrorString(e));
        cudaGetLastError();
        return MG_ERR_OOM;
    }
    ctx->allocs.push_back(q);
    e = cudaMemsetAsync(q, 0, count * sizeof(T), ctx->st);
    if (e != cudaSuccess) {
        set_err("cudaMemsetAsync failed: %s", cudaGetErrorString(e));
        return MG_ERR_CUDA;
    }
    *p = (T *)q;
    return MG_OK;
}

bool can_coarsen(const Dims &d) {
    const int n[3] = {d.nx, d.ny, d.nz};
    for (int a = 0; a < 3; a++)
        if (n[a] % 2 != 0 || n[a] / 2 < 4) return false;
    return true;
}

size_t corner_count(const Dims &d) { return 3 * (size_t)d.cs; }

// ---------------------------------------------------------------- timers

// fold completed event pairs into the totals (the stream must be idle)
mg_status prof_drain(mg_ctx *ctx) {
    for (int i = 0; i < ctx->npend; i++) {
        float ms = 0.f;
        CK(cudaEventElapsedTime(&ms, ctx->pend_ev[i][0], ctx->pend_ev[i][1]));
        ctx->prof_ms += ms;
        ctx->prof_sweeps += ctx->pend_sweeps[i];
        ctx->prof_launches += ctx->pend_launches[i];
    }
    ctx->npend = 0;
    return MG_OK;
}

// ---------------------------------------------------------------- norms

// ||r||^2 from the partial sums of the last reduction kernel
// the fused sweep's error word (set when a bounded wait for a neighbouring
// tile gave up), read after the stream has drained; cleared when reported
mg_status sync_error(mg_ctx *ctx) {
    if (!ctx->has_sync || !*ctx->herr) return MG_OK;
    *ctx->herr = 0;
    CK(cudaMemsetAsync(ctx->sync.err, 0, sizeof(int), ctx->st));
    set_err("fused Gauss-Seidel sweep: a wait for a neighbouring tile gave up");
    return MG_ERR_CUDA;
}

mg_status read_sum(mg_ctx *ctx, double *out) {
    CK(sum_partials(ctx->partials, ctx->dsum, ctx->st));
    CK(cudaMemcpyAsync(ctx->hsum, ctx->dsum, sizeof(double), cudaMemcpyDeviceToHost, ctx->st));
    if (ctx->has_sync)
        CK(cudaMemcpyAsync(ctx->herr, ctx->sync.err, sizeof(int), cudaMemcpyDeviceToHost, ctx->st));
    CK(cudaStreamSynchronize(ctx->st));
    *out = ctx->hsum[0];
    CKS(sync_error(ctx));
    return prof_drain(ctx);
}

// ||b - A v||_2 on the finest level (FP64), optionally writing
// float(r * out_scale) into r32; wall_only gives ||b_lifted||_2
mg_status fine_resnorm(mg_ctx *ctx, const double *b, const double *v, bool wall_only, float *r32,
                       double out_scale, double *norm, int split32 = 0) {
    CK(residual_norm_fine64(ctx->L[0], ctx->f64, b, v, wall_only, r32, out_scale, ctx->partials,
                            ctx->st, split32));
    double s2;
    CKS(read_sum(ctx, &s2));
    *norm = sqrt(s2);
    return MG_OK;
}

// ---------------------------------------------------------------- V-cycles

template <typename T>
struct Bufs;
template <>
struct Bufs<double> {
    static double *x(mg_ctx *c, int l) { return c->x64[l]; }
    static double *b(mg_ctx *c, int l) { return c->b64[l]; }
    static double *r(mg_ctx *c, int l) { return c->r64[l]; }
    static const Fine<double> &fine(mg_ctx *c) { return c->f64; }
    static const Coarse<double> &coarse(mg_ctx *c, int l) { return c->c64[l]; }
};
template <>
struct Bufs<float> {
    static float *x(mg_ctx *c, int l) { return c->x32[l]; }
    static float *b(mg_ctx *c, int l) { return c->b32[l]; }
    static float *r(mg_ctx *c, int l) { return c->r32[l]; }
    static const Fine<float> &fine(mg_ctx *c) { return c->f32; }
    static const Coarse<float> &coarse(mg_ctx *c, int l) { return c->c32[l]; }
};

template <typename T>
mg_status gs_pass(mg_ctx *ctx, int l, const T *b, T *x, int colour) {
    if (l == 0)
        CK(gs_colour_fine(ctx->L[0], Bufs<T>::fine(ctx), b, x, colour, ctx->st));
    else
        CK(gs_colour_coarse(ctx->L[l], Bufs<T>::coarse(ctx, l), b, x, colour, ctx->st));
    return MG_OK;
}

// FP32 sweeps on level l with the tiled two-phase kernels, ping-ponging
// between x and the level's partner buffer (whose wall planes are made equal
// to x's; the solver's own level arrays and partners all keep zero walls)
mg_status sweeps_tiled(mg_ctx *ctx, int l, const float *b, float *x, int sweeps, bool descending) {
    const Dims &d = ctx->L[l];
    float *a = x, *o = ctx->xs32[l];
    if (x != ctx->x32[l]) {
        const size_t plane = (size_t)d.ny * d.nx;
        for (int c = 0; c < 3; c++) {
            CK(cudaMemcpyAsync(o + c * d.cs, x + c * d.cs, plane * sizeof(float),
                               cudaMemcpyDeviceToDevice, ctx->st));
            CK(cudaMemcpyAsync(o + c * d.cs + d.nz * plane, x + c * d.cs + d.nz * plane,
                               plane * sizeof(float), cudaMemcpyDeviceToDevice, ctx->st));
        }
    }
    for (int s = 0; s < sweeps; s++) {
        if (l == 0)
            CK(gs_sweep_fine_tiled(d, ctx->f32, b, a, o, descending, ctx->st, ctx->split0,
                                   ctx->has_sync ? &ctx->sync : nullptr));
        else
            CK(gs_sweep_coarse_tiled(d, ctx->c32[l], b, a, o, descending, ctx->st));
        float *t = a;
        a = o;
        o = t;
    }
    if (a != x)
        CK(cudaMemcpyAsync(x, a, 3 * (size_t)d.cs * sizeof(float), cudaMemcpyDeviceToDevice,
                           ctx->st));
    if (x != ctx->x32[l]) {
        // the partner holds x's walls; restore the solver's zero walls
        const size_t plane = (size_t)d.ny * d.nx;
        for (int c = 0; c < 3; c++) {
            CK(cudaMemsetAsync(ctx->xs32[l] + c * d.cs, 0, plane * sizeof(float), ctx->st));
            CK(cudaMemsetAsync(ctx->xs32[l] + c * d.cs + d.nz * plane, 0, plane * sizeof(float),
                               ctx->st));
        }
    }
    return MG_OK;
}

template <typename T>
mg_status sweeps_colour(mg_ctx *ctx, int l, const T *b, T *x, int sweeps, bool descending) {
    for (int s = 0; s < sweeps; s++)
        for (int c = 0; c < 8; c++) CKS(gs_pass<T>(ctx, l, b, x, descending ? 7 - c : c));
    return MG_OK;
}

template <typename T>
mg_status sweeps(mg_ctx *ctx, int l, const T *b, T *x, int n, bool descending) {
    return sweeps_colour<T>(ctx, l, b, x, n, descending);
}

// FP32: the two-phase kernels (row strips where the rows fit, else tiles),
// except on large coarse levels without row strips, where the 27-point tile
// kernel (128 registers, 2 CTAs per SM) loses to colour launches (measured on
// GB300 at 128^2 planes: 71 us per phase launch against 4 x 13 us)
template <>
mg_status sweeps<float>(mg_ctx *ctx, int l, const float *b, float *x, int n, bool descending) {
    const Dims &d = ctx->L[l];
    const bool colour = (ctx->opts.flags & MG_FLAG_COLOUR_PASSES) ||
                        (l > 0 && (long)d.nx * d.ny >= 128L * 128L && !coarse_rows_fit(d));
    if (!colour) return sweeps_tiled(ctx, l, b, x, n, descending);
    return sweeps_colour<float>(ctx, l, b, x, n, descending);
}

// queue one timed event pair for the next drain
mg_status prof_push(mg_ctx *ctx, cudaEvent_t e0, cudaEvent_t e1, long sweeps, long launches) {
    if (ctx->npend == kProfSlots) {
        CK(cudaStreamSynchronize(ctx->st));
        CKS(prof_drain(ctx));
    }
    ctx->pend_ev[ctx->npend][0] = e0;
    ctx->pend_ev[ctx->npend][1] = e1;
    ctx->pend_sweeps[ctx->npend] = sweeps;
    ctx->pend_launches[ctx->npend] = launches;
    ctx->npend++;
    return MG_OK;
}

template <typename T>
mg_status smooth(mg_ctx *ctx, int l, const T *b, T *x, int sweeps_n, bool descending) {
    InnerGraph *G = ctx->capturing;
    const bool timed = l == 0 && sweeps_n > 0 &&
                       (G ? G->nev < 2 * kMaxInner : ctx->prof_on);
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (timed && !G) {
        if (ctx->npend == kProfSlots) {
            CK(cudaStreamSynchronize(ctx->st));
            CKS(prof_drain(ctx));
        }
        e0 = ctx->ev[ctx->npend][0];
        e1 = ctx->ev[ctx->npend][1];
    } else if (timed) {
        e0 = G->ev[G->nev][0];
        e1 = G->ev[G->nev][1];
    }
    // inside a capture an external record node is needed for the replay to
    // take a timestamp (a plain record only marks a capture position)
    const unsigned rec = G ? cudaEventRecordExternal : cudaEventRecordDefault;
    const long launches0 = g_launches.load();
    if (timed) CK(cudaEventRecordWithFlags(e0, ctx->st, rec));
    CKS(sweeps<T>(ctx, l, b, x, sweeps_n, descending));
    if (timed) {
        CK(cudaEventRecordWithFlags(e1, ctx->st, rec));
        const long nl = g_launches.load() - launches0;
        if (G) {
            G->sweeps[G->nev] = sweeps_n;
            G->launches[G->nev] = nl;
            G->nev++;
        } else {
            CKS(prof_push(ctx, e0, e1, sweeps_n, nl));
        }
    }
    return MG_OK;
}

// the solver's FP32 finest-level arrays may be in parity-split column order
template <typename T>
int split_of(const mg_ctx *ctx, int l) {
    return 0;
}
template <>
int split_of<float>(const mg_ctx *ctx, int l) {
    return l == 0 ? ctx->split0 : 0;
}

template <typename T>
mg_status residual_level(mg_ctx *ctx, int l, const T *b, const T *x, T *r) {
    if (l == 0)
        CK(residual_fine(ctx->L[0], Bufs<T>::fine(ctx), b, x, r, ctx->st));
    else
        CK(residual_coarse(ctx->L[l], Bufs<T>::coarse(ctx, l), b, x, r, ctx->st));
    return MG_OK;
}

template <>
mg_status residual_level<float>(mg_ctx *ctx, int l, const float *b, const float *x, float *r) {
    if (l == 0)
        CK(residual_fine(ctx->L[0], ctx->f32, b, x, r, ctx->st, ctx->split0));
    else
        CK(residual_coarse(ctx->L[l], ctx->c32[l], b, x, r, ctx->st));
    return MG_OK;
}

inline cudaError_t restrict_fw_any(const Dims &d, const double *r, double *bc, cudaStream_t s,
                                   int) {
    return restrict_fw(d, r, bc, s);
}
inline cudaError_t restrict_fw_any(const Dims &d, const float *r, float *bc, cudaStream_t s,
                                   int split) {
    return restrict_fw(d, r, bc, s, split);
}
inline cudaError_t prolong_add_any(const Dims &d, const double *xc, double *x, cudaStream_t s,
                                   int) {
    return prolong_add(d, xc, x, s);
}
inline cudaError_t prolong_add_any(const Dims &d, const float *xc, float *x, cudaStream_t s,
                                   int split) {
    return prolong_add(d, xc, x, s, split);
}

// bc = T^T (b - A_l x) on level l; r is level l's residual buffer
template <typename T>
mg_status residual_restrict_level(mg_ctx *ctx, int l, const T *b, const T *x, T *r, T *bc) {
    CKS(residual_level<T>(ctx, l, b, x, r));
    CK(restrict_fw_any(ctx->L[l], r, bc, ctx->st, split_of<T>(ctx, l)));
    return MG_OK;
}

// FP32 finest level: residual and restriction fused where the row-strip
// kernel takes the grid (the residual is never stored; r receives the
// per-plane partial sums), else the two passes
template <>
mg_status residual_restrict_level<float>(mg_ctx *ctx, int l, const float *b, const float *x,
                                         float *r, float *bc) {
    if (l == 0 && !(ctx->opts.flags & MG_FLAG_UNFUSED_TRANSFERS)) {
        const cudaError_t e =
            residual_restrict_fine_rows(ctx->L[0], ctx->f32, b, x, r, bc, ctx->st, ctx->split0);
        if (e == cudaSuccess) return MG_OK;
        if (e != cudaErrorNotSupported) CK(e);
    }
    CKS(residual_level<float>(ctx, l, b, x, r));
    CK(restrict_fw_any(ctx->L[l], r, bc, ctx->st, split_of<float>(ctx, l)));
    return MG_OK;
}

// one V-cycle for A_l x = b on level l (section 3.6)
template <typename T>
mg_status vcycle(mg_ctx *ctx, int l, const T *b, T *x) {
    T *r = Bufs<T>::r(ctx, l);
    if (l == ctx->nlev - 1) {
        CKS(residual_level<T>(ctx, l, b, x, r));
        CK(coarse_solve(ctx->L[l], ctx->Ainv, ctx->ncoarse, r, x, ctx->st));
        return MG_OK;
    }
    CKS(smooth<T>(ctx, l, b, x, ctx->opts.nu1, false));
    T *bc = Bufs<T>::b(ctx, l + 1), *xc = Bufs<T>::x(ctx, l + 1);
    CKS(residual_restrict_level<T>(ctx, l, b, x, r, bc));
    CK(cudaMemsetAsync(xc, 0, corner_count(ctx->L[l + 1]) * sizeof(T), ctx->st));
    CKS(vcycle<T>(ctx, l + 1, bc, xc));
    CK(prolong_add_any(ctx->L[l], xc, x, ctx->st, split_of<T>(ctx, l)));
    CKS(smooth<T>(ctx, l, b, x, ctx->opts.nu2, true));
    return MG_OK;
}

mg_status check_ctx(mg_ctx *ctx) {
    if (!ctx) {
        set_err("null context");
        return MG_ERR_ARG;
    }
    if (ctx->broken) {
        set_err("context unusable after an earlier CUDA failure");
        return MG_ERR_STATE;
    }
    return MG_OK;
}

mg_status solve_fp64(mg_ctx *ctx, const double *b, double *v, double tol, mg_stats *st) {
    double bn, rn;
    CKS(fine_resnorm(ctx, b, v, true, nullptr, 0.0, &bn));
    st->bnorm = bn;
    if (bn == 0.0) {
        CK(zero_interior(ctx->L[0], v, ctx->st));
        st->rel_resid = 0.0;
        st->resid_hist[0] = 0.0;
        return MG_OK;
    }
    CKS(fine_resnorm(ctx, b, v, false, nullptr, 0.0, &rn));
    double rel = rn / bn;
    st->resid_hist[0] = rel;
    int it = 0;
    for (;;) {
        st->rel_resid = rel;
        st->cycles = st->outer_iters = it;
        if (!isfinite(rel)) {
            set_err("non-finite residual after %d cycles", it);
            return MG_ERR_NONFINITE;
        }
        if (tol > 0.0 && rel <= tol) return MG_OK;
        if (it >= ctx->opts.max_cycles) {
            if (tol > 0.0) {
                set_err("no convergence: relative residual %.3e after %d cycles", rel, it);
                return MG_ERR_NOCONV;
            }
            return MG_OK;
        }
        CKS(vcycle<double>(ctx, 0, b, v));
        it++;
        CKS(fine_resnorm(ctx, b, v, false, nullptr, 0.0, &rn));
        rel = rn / bn;
        if (it < MG_HIST) st->resid_hist[it] = rel;
    }
}

// FP32 V-cycles on the correction equation inside FP64 iterative refinement:
//   r = b - A v (FP64, stored as float(r / s)), e ~ A^{-1} r by FP32 V-cycles
//   from e = 0, v += s e.
// With opts.inner_cycles > 0 every refinement step runs that many cycles.
// With 0 the count is chosen per step: enough cycles to bring the FP64
// residual to tol at the contraction factor observed so far (initially 0.4),
// at least 1 and at most kMaxInner, so that few FP64 residuals are needed.

int inner_count(const mg_ctx *ctx, double rel, double tol, double kappa) {
    if (ctx->opts.inner_cycles > 0) return ctx->opts.inner_cycles;
    if (!(tol > 0.0) || !(rel > tol)) return kMaxInner;
    const double need = log(0.7 * tol / rel) / log(kappa);
    int n = (int)ceil(need);
    return n < 1 ? 1 : (n > kMaxInner ? kMaxInner : n);
}

// n FP32 V-cycles on the finest correction equation from e = 0
mg_status inner_cycles_direct(mg_ctx *ctx, int n) {
    CK(cudaMemsetAsync(ctx->x32[0], 0, corner_count(ctx->L[0]) * sizeof(float), ctx->st));
    for (int c = 0; c < n; c++) CKS(vcycle<float>(ctx, 0, ctx->b32[0], ctx->x32[0]));
    return MG_OK;
}

// the same as one CUDA graph: captured on the private stream at first use,
// replayed on the context's stream
mg_status inner_cycles(mg_ctx *ctx, int n) {
    if (ctx->opts.flags & MG_FLAG_NO_GRAPH) return inner_cycles_direct(ctx, n);
    InnerGraph *G = ctx->graphs[n];
    if (!G) {
        G = new InnerGraph();
        ctx->graphs[n] = G;
        for (int i = 0; i < 2 * kMaxInner; i++) {
            CK(cudaEventCreate(&G->ev[i][0]));
            CK(cudaEventCreate(&G->ev[i][1]));
        }
        cudaStream_t user = ctx->st;
        const long k0 = g_launches.load();
        CK(cudaStreamBeginCapture(ctx->cap, cudaStreamCaptureModeThreadLocal));
        ctx->st = ctx->cap;
        ctx->capturing = G;
        const mg_status body = inner_cycles_direct(ctx, n);
        ctx->capturing = nullptr;
        ctx->st = user;
        cudaGraph_t graph = nullptr;
        const cudaError_t ee = cudaStreamEndCapture(ctx->cap, &graph);
        G->kernels = g_launches.load() - k0;
        g_launches.fetch_sub(G->kernels);  // counted when replayed, not when captured
        if (body != MG_OK) {
            if (graph) cudaGraphDestroy(graph);
            return body;
        }
        CK(ee);
        const cudaError_t ei = cudaGraphInstantiate(&G->exec, graph, 0);
        cudaGraphDestroy(graph);
        CK(ei);
    }
    CK(cudaGraphLaunch(G->exec, ctx->st));
    count_launch(G->kernels);
    if (ctx->prof_on)
        for (int i = 0; i < G->nev; i++)
            CKS(prof_push(ctx, G->ev[i][0], G->ev[i][1], G->sweeps[i], G->launches[i]));
    return MG_OK;
}

mg_status solve_mixed(mg_ctx *ctx, const double *b, double *v, double tol, mg_stats *st) {
    double bn, rn;
    CKS(fine_resnorm(ctx, b, v, true, nullptr, 0.0, &bn));
    st->bnorm = bn;
    if (bn == 0.0) {
        CK(zero_interior(ctx->L[0], v, ctx->st));
        st->rel_resid = 0.0;
        st->resid_hist[0] = 0.0;
        return MG_OK;
    }
    double scale = bn;
    CKS(fine_resnorm(ctx, b, v, false, ctx->b32[0], 1.0 / scale, &rn, ctx->split0));
    double rel = rn / bn;
    st->resid_hist[0] = rel;
    int outer = 0, cycles = 0;
    double kappa = 0.4;  // V-cycle contraction estimate, refined from the history
    for (;;) {
        st->rel_resid = rel;
        st->cycles = cycles;
        st->outer_iters = outer;
        if (!isfinite(rel)) {
            set_err("non-finite residual after %d refinement steps", outer);
            return MG_ERR_NONFINITE;
        }
        if (tol > 0.0 && rel <= tol) return MG_OK;
        if (outer >= ctx->opts.max_cycles) {
            if (tol > 0.0) {
                set_err("no convergence: relative residual %.3e after %d refinement steps", rel,
                        outer);
                return MG_ERR_NOCONV;
            }
            return MG_OK;
        }
        const int n = inner_count(ctx, rel, tol, kappa);
        CKS(inner_cycles(ctx, n));
        CK(axpy_f32(ctx->L[0], scale, ctx->x32[0], v, ctx->st, ctx->split0));
        outer++;
        cycles += n;
        scale = rn;
        CKS(fine_resnorm(ctx, b, v, false, ctx->b32[0], 1.0 / scale, &rn, ctx->split0));
        const double rel_new = rn / bn;
        if (rel_new > 0.0 && rel_new < rel) {
            const double k = pow(rel_new / rel, 1.0 / n);
            kappa = k < 0.05 ? 0.05 : (k > 0.9 ? 0.9 : k);
        }
        rel = rel_new;
        if (outer < MG_HIST) st->resid_hist[outer] = rel;
    }
}

StepParams step_params(const mg_ctx *ctx, double dt) {
    StepParams p;
    p.nx = ctx->L[0].nx;
    p.ny = ctx->L[0].ny;
    p.nz = ctx->L[0].nz;
    p.h = ctx->h;
    p.dt = dt;
    p.lam = ctx->lam;
    p.mu = ctx->mu;
    const stz_params &z = ctx->stz;
    p.tau0 = z.tau0;
    p.eps0 = z.eps0;
    p.c0 = z.c0;
    p.Delta_K = z.Delta_K;
    p.Omega = z.Omega;
    p.T = z.T;
    p.chi_inf = z.chi_inf;
    p.ez_K = z.ez_K;
    p.sY = z.sY;
    p.l = z.l;
    p.kB = z.kB;
    return p;
}

WallParams wall_params(const mg_ctx *ctx, double t) {
    WallParams w;
    w.nx = ctx->L[0].nx;
    w.ny = ctx->L[0].ny;
    w.nz = ctx->L[0].nz;
    w.kind = ctx->bc.kind;
    w.h = ctx->h;
    w.t = t;
    w.U_B = ctx->bc.U_B;
    w.t_ramp = ctx->bc.t_ramp;
    w.omega = ctx->bc.omega;
    w.R = ctx->bc.R;
    w.lambda_w = ctx->bc.lambda_w;
    return w;
}

}  // namespace

// ======================================================================= ABI

extern "C" {

const char *mg_status_str(mg_status s) {
    switch (s) {
    case MG_OK: return "ok";
    case MG_ERR_ARG: return "invalid argument";
    case MG_ERR_SHAPE: return "unsupported grid shape";
    case MG_ERR_CUDA: return "CUDA error";
    case MG_ERR_OOM: return "out of device memory";
    case MG_ERR_NOCONV: return "not converged";
    case MG_ERR_NONFINITE: return "non-finite residual";
    case MG_ERR_STATE: return "context unusable";
    }
    return "unknown status";
}

const char *mg_last_error(void) { return g_err; }

void mg_free(mg_ctx *ctx) {
    if (!ctx) return;
    if (ctx->st) cudaStreamSynchronize(ctx->st);
    else cudaDeviceSynchronize();
    for (void *p : ctx->allocs) cudaFree(p);
    if (ctx->hsum) cudaFreeHost(ctx->hsum);
    if (ctx->herr) cudaFreeHost(ctx->herr);
    if (ctx->prof_events)
        for (int i = 0; i < kProfSlots; i++) {
            cudaEventDestroy(ctx->ev[i][0]);
            cudaEventDestroy(ctx->ev[i][1]);
        }
    for (int n = 0; n <= kMaxInner; n++) {
        InnerGraph *G = ctx->graphs[n];
        if (!G) continue;
        if (G->exec) cudaGraphExecDestroy(G->exec);
        for (int i = 0; i < 2 * kMaxInner; i++) {
            if (G->ev[i][0]) cudaEventDestroy(G->ev[i][0]);
            if (G->ev[i][1]) cudaEventDestroy(G->ev[i][1]);
        }
        delete G;
    }
    if (ctx->cap) cudaStreamDestroy(ctx->cap);
    delete ctx;
}

mg_status mg_setup(const mg_grid *grid, const mg_moduli *moduli, const mg_bc *bc,
                   const stz_params *stz, const mg_opts *opts, void *stream, mg_ctx **out) {
    mg_ctx *ctx = nullptr;
    if (!grid || !moduli || !opts || !out) {
        set_err("mg_setup: null argument");
        return MG_ERR_ARG;
    }
    *out = nullptr;
    const int nx = grid->nx, ny = grid->ny, nz = grid->nz;
    if (nx < 4 || ny < 4 || nz < 2 || nx % 2 || ny % 2 || nz % 2) {
        set_err("mg_setup: grid %dx%dx%d unsupported (nx, ny even >= 4; nz even >= 2)", nx, ny, nz);
        return MG_ERR_SHAPE;
    }
    if (!(grid->h > 0.0) || !(moduli->mu > 0.0) || !(moduli->K - 2.0 * moduli->mu / 3.0 + moduli->mu > 0.0)) {
        set_err("mg_setup: need h > 0, mu > 0 and lambda + mu > 0");
        return MG_ERR_ARG;
    }
    if (opts->precision != MG_FP64 && opts->precision != MG_MIXED) {
        set_err("mg_setup: precision must be MG_FP64 or MG_MIXED");
        return MG_ERR_ARG;
    }
    if (opts->nu1 < 0 || opts->nu2 < 0 || opts->max_cycles < 0 || opts->max_cycles >= MG_HIST ||
        opts->inner_cycles < 0 || opts->inner_cycles > kMaxInner) {
        set_err("mg_setup: bad nu1/nu2/max_cycles/inner_cycles");
        return MG_ERR_ARG;
    }
    ctx = new mg_ctx();  // value-initialised: every pointer and flag starts at zero
    ctx->st = (cudaStream_t)stream;
    ctx->opts = *opts;
    ctx->h = grid->h;
    ctx->mu = moduli->mu;
    ctx->lam = moduli->K - 2.0 * moduli->mu / 3.0;
    if (bc) {
        ctx->bc = *bc;
        ctx->has_bc = true;
    }
    if (stz) {
        ctx->stz = *stz;
        ctx->has_stz = true;
    }
    // hierarchy
    ctx->L[0] = make_dims(nx, ny, nz);
    ctx->nlev = 1;
    while (ctx->nlev < kMaxLev && can_coarsen(ctx->L[ctx->nlev - 1])) {
        const Dims &p = ctx->L[ctx->nlev - 1];
        ctx->L[ctx->nlev] = make_dims(p.nx / 2, p.ny / 2, p.nz / 2);
        ctx->nlev++;
    }
    const Dims &dc = ctx->L[ctx->nlev - 1];
    const long nco = 3L * dc.nx * dc.ny * (dc.nz - 1);
    if (nco > kMaxCoarse) {
        set_err("mg_setup: coarsest level %dx%dx%d has %ld unknowns (> %d)", dc.nx, dc.ny, dc.nz,
                nco, kMaxCoarse);
        delete ctx;
        return MG_ERR_SHAPE;
    }
    ctx->ncoarse = (int)nco;
    // finest FP32 arrays in parity-split order when the tiled sweeps run on a
    // grid with coarser levels (so level 0 is never the directly solved one)
    ctx->split0 = (ctx->nlev > 1 && !(opts->flags & MG_FLAG_COLOUR_PASSES)) ? 1 : 0;
    fine_table(ctx->lam, ctx->mu, ctx->S[0]);
    for (int l = 1; l < ctx->nlev; l++) galerkin_table(ctx->S[l - 1], ctx->S[l]);
    const double lp = (ctx->lam + 2.0 * ctx->mu) / ctx->mu, kq = (ctx->lam + ctx->mu) / (4.0 * ctx->mu);
    ctx->f64.d0 = 2.0 * lp + 4.0;
    ctx->f64.lp = lp;
    ctx->f64.kq = kq;
    ctx->f64.dinv = 1.0 / ctx->f64.d0;
    ctx->f32.d0 = (float)ctx->f64.d0;
    ctx->f32.lp = (float)lp;
    ctx->f32.kq = (float)kq;
    ctx->f32.dinv = (float)ctx->f64.dinv;
    for (int l = 0; l < ctx->nlev; l++) {
        if (!parity_classes(ctx->S[l], ctx->c64[l])) {
            set_err("mg_setup: the level-%d operator lacks the reflection symmetry of its "
                    "parity-class form, or has a singular centre block", l);
            delete ctx;
            return MG_ERR_ARG;
        }
        const Coarse<double> &c = ctx->c64[l];
        Coarse<float> &f = ctx->c32[l];
        for (int a = 0; a < 3; a++) {
            for (int m = 0; m < 8; m++) f.cd[a][m] = (float)c.cd[a][m];
            for (int m = 0; m < 2; m++) f.g[a][m] = (float)c.g[a][m];
            f.dinv[a] = (float)c.dinv[a];
        }
    }
    std::vector<double> Ainv;
    if (!coarse_inverse(dc, ctx->S[ctx->nlev - 1], Ainv)) {
        set_err("mg_setup: coarsest operator is not positive definite");
        delete ctx;
        return MG_ERR_ARG;
    }
    {
        cudaError_t e = smoother_init();
        if (e == cudaSuccess) e = plane_init();
        if (e != cudaSuccess) {
            set_err("mg_setup: %s", cudaGetErrorString(e));
            delete ctx;
            return MG_ERR_CUDA;
        }
    }
    // buffers
    mg_status s = MG_OK;
#define ALLOC(p, n)                      \
    do {                                 \
        s = dalloc(ctx, &(p), (n));      \
        if (s != MG_OK) goto fail;       \
    } while (0)
    for (int l = 0; l < ctx->nlev; l++) {
        const size_t n = corner_count(ctx->L[l]);
        if (l > 0) {
            ALLOC(ctx->x64[l], n);
            ALLOC(ctx->b64[l], n);
        }
        ALLOC(ctx->r64[l], n);
        ALLOC(ctx->x32[l], n);
        ALLOC(ctx->b32[l], n);
        ALLOC(ctx->r32[l], n);
        ALLOC(ctx->xs32[l], n);
    }
    ALLOC(ctx->Ainv, Ainv.size());
    ALLOC(ctx->partials, (size_t)kRedBlocks);
    ALLOC(ctx->dsum, (size_t)1);
    {
        const size_t nc = (size_t)nx * ny * nz;
        ALLOC(ctx->sig_star, 6 * nc);
        ALLOC(ctx->dpl, nc);
        ALLOC(ctx->sbar, nc);
        ALLOC(ctx->chi_tmp, nc);
        ALLOC(ctx->rhs, corner_count(ctx->L[0]));
    }
    {
        long na = 0;
        if ((opts->flags & MG_FLAG_FUSED_SWEEP) && !(opts->flags & MG_FLAG_COLOUR_PASSES) &&
            ctx->nlev > 1 &&
            fused_sweep_sizes(ctx->L[0], na)) {
            ALLOC(ctx->sync.aflag, (size_t)na);
            ALLOC(ctx->sync.epoch, (size_t)1);
            ALLOC(ctx->sync.done, (size_t)1);
            ALLOC(ctx->sync.err, (size_t)1);
            if (cudaMallocHost((void **)&ctx->herr, sizeof(int)) != cudaSuccess) {
                set_err("cudaMallocHost failed");
                s = MG_ERR_OOM;
                goto fail;
            }
            *ctx->herr = 0;
            ctx->has_sync = true;
        }
    }
#undef ALLOC
    if (cudaStreamCreateWithFlags(&ctx->cap, cudaStreamNonBlocking) != cudaSuccess) {
        set_err("cudaStreamCreateWithFlags failed");
        s = MG_ERR_CUDA;
        goto fail;
    }
    if (cudaMallocHost((void **)&ctx->hsum, sizeof(double)) != cudaSuccess) {
        set_err("cudaMallocHost failed");
        s = MG_ERR_OOM;
        goto fail;
    }
    if (cudaMemcpyAsync(ctx->Ainv, Ainv.data(), Ainv.size() * sizeof(double),
                        cudaMemcpyHostToDevice, ctx->st) != cudaSuccess ||
        cudaStreamSynchronize(ctx->st) != cudaSuccess) {
        set_err("mg_setup: upload failed: %s", cudaGetErrorString(cudaGetLastError()));
        s = MG_ERR_CUDA;
        goto fail;
    }
    *out = ctx;
    return MG_OK;
fail:
    mg_free(ctx);
    return s;
}

mg_status mg_solve(mg_ctx *ctx, const double *rhs, double *v, double tol, mg_stats *stats) {
    CKS(check_ctx(ctx));
    if (!rhs || !v) {
        set_err("mg_solve: null array");
        return MG_ERR_ARG;
    }
    mg_stats local;
    mg_stats *st = stats ? stats : &local;
    memset(st, 0, sizeof(*st));
    if (ctx->opts.precision == MG_FP64) return solve_fp64(ctx, rhs, v, tol, st);
    return solve_mixed(ctx, rhs, v, tol, st);
}

mg_status qs_run(mg_ctx *ctx, qs_state *state, int nsteps, double dt, double tol,
                 mg_stats *stats) {
    CKS(check_ctx(ctx));
    if (!state || !state->v || !state->sigma || !state->chi || !(dt > 0.0) || nsteps < 0) {
        set_err("qs_run: null state array, dt <= 0 or nsteps < 0");
        return MG_ERR_ARG;
    }
    if (!ctx->has_stz || !ctx->has_bc) {
        set_err("qs_run: context was set up without stz/bc parameters");
        return MG_ERR_ARG;
    }
    if (nsteps == 0) return MG_OK;
    const StepParams p = step_params(ctx, dt);
    const bool advect = (ctx->opts.flags & MG_FLAG_ADVECT_STRESS) != 0;
    CK(stress_predict(p, state->v, state->sigma, state->chi, ctx->sig_star, ctx->dpl, ctx->sbar,
                      ctx->st));
    mg_status s = MG_OK;
    for (int n = 0; n < nsteps; n++) {
        // the previous step's correction and this step's predictor share v
        if (n > 0)
            CK(correct_predict(p, state->v, ctx->sig_star, state->sigma, ctx->chi_tmp, state->chi,
                               ctx->dpl, ctx->sbar, ctx->st));
        // optional -(u.grad) sigma^n in sigma* (state->sigma and v hold step n)
        if (advect) CK(stress_advect(p, state->v, state->sigma, ctx->sig_star, ctx->st));
        CK(chi_update(p, state->sigma, state->chi, ctx->dpl, ctx->sbar, ctx->chi_tmp, ctx->st));
        CK(wall_fill(wall_params(ctx, state->t + dt), state->v, ctx->st));
        CK(div_rhs(p, ctx->sig_star, ctx->rhs, ctx->st));
        s = mg_solve(ctx, ctx->rhs, state->v, tol, stats ? stats + n : nullptr);
        if (s == MG_ERR_CUDA || s == MG_ERR_STATE || s == MG_ERR_ARG) return s;
        state->t += dt;
        state->step += 1;
        if (s != MG_OK) break;  // advance this step with the last iterate, then stop
    }
    CK(stress_correct(p, state->v, ctx->sig_star, state->sigma, ctx->chi_tmp, state->chi, ctx->st));
    CK(cudaStreamSynchronize(ctx->st));
    return s;
}

mg_status qs_step(mg_ctx *ctx, qs_state *state, double dt, double tol, mg_stats *stats) {
    return qs_run(ctx, state, 1, dt, tol, stats);
}

mg_status qs_explicit_step(mg_ctx *ctx, qs_state *state, double dt, double rho, double kappa,
                           int nsteps) {
    CKS(check_ctx(ctx));
    if (!state || !state->v || !state->sigma || !state->chi || !(dt > 0.0) || !(rho > 0.0) ||
        !(kappa >= 0.0) || nsteps < 0) {
        set_err("qs_explicit_step: null state array, dt <= 0, rho <= 0, kappa < 0 or nsteps < 0");
        return MG_ERR_ARG;
    }
    if (!ctx->has_stz || !ctx->has_bc) {
        set_err("qs_explicit_step: context was set up without stz/bc parameters");
        return MG_ERR_ARG;
    }
    const Dims &d = ctx->L[0];
    const size_t nc = (size_t)d.nx * d.ny * d.nz, nv = corner_count(d);
    const StepParams p = step_params(ctx, dt);
    // the new stress, chi and velocity go to the context's step scratch
    // (sig_star, chi_tmp, rhs), then back into the state
    for (int n = 0; n < nsteps; n++) {
        CK(explicit_stress(p, state->v, state->sigma, state->chi, ctx->sig_star, ctx->dpl,
                           ctx->sbar, ctx->st));
        CK(chi_update(p, state->sigma, state->chi, ctx->dpl, ctx->sbar, ctx->chi_tmp, ctx->st));
        CK(explicit_velocity(p, rho, kappa, state->v, state->sigma, ctx->rhs, ctx->st));
        CK(cudaMemcpyAsync(state->sigma, ctx->sig_star, 6 * nc * sizeof(double),
                           cudaMemcpyDeviceToDevice, ctx->st));
        CK(cudaMemcpyAsync(state->chi, ctx->chi_tmp, nc * sizeof(double),
                           cudaMemcpyDeviceToDevice, ctx->st));
        CK(cudaMemcpyAsync(state->v, ctx->rhs, nv * sizeof(double), cudaMemcpyDeviceToDevice,
                           ctx->st));
        CK(wall_fill(wall_params(ctx, state->t + dt), state->v, ctx->st));
        state->t += dt;
        state->step += 1;
    }
    CK(cudaStreamSynchronize(ctx->st));
    return MG_OK;
}

// ------------------------------------------------------------ components

int mg_num_levels(const mg_ctx *ctx) { return ctx ? ctx->nlev : 0; }

mg_status mg_level_dims(const mg_ctx *ctx, int level, int *dims) {
    if (!ctx || !dims || level < 0 || level >= ctx->nlev) {
        set_err("mg_level_dims: bad argument");
        return MG_ERR_ARG;
    }
    dims[0] = ctx->L[level].nx;
    dims[1] = ctx->L[level].ny;
    dims[2] = ctx->L[level].nz;
    return MG_OK;
}

mg_status mg_level_stencil(const mg_ctx *ctx, int level, double *host_S) {
    if (!ctx || !host_S || level < 0 || level >= ctx->nlev) {
        set_err("mg_level_stencil: bad argument");
        return MG_ERR_ARG;
    }
    memcpy(host_S, ctx->S[level], 243 * sizeof(double));
    return MG_OK;
}

static mg_status level_arg(mg_ctx *ctx, int level, int need_coarser) {
    CKS(check_ctx(ctx));
    if (level < 0 || level >= ctx->nlev - (need_coarser ? 1 : 0)) {
        set_err("bad level %d", level);
        return MG_ERR_ARG;
    }
    return MG_OK;
}

mg_status mg_residual(mg_ctx *ctx, int level, const double *b, const double *x, double *r) {
    CKS(level_arg(ctx, level, 0));
    if (!b || !x || !r || r == x) {
        set_err("mg_residual: bad arrays");
        return MG_ERR_ARG;
    }
    CKS(residual_level<double>(ctx, level, b, x, r));
    CK(cudaStreamSynchronize(ctx->st));
    return MG_OK;
}

mg_status mg_residual32(mg_ctx *ctx, int level, const float *b, const float *x, float *r) {
    CKS(level_arg(ctx, level, 0));
    if (!b || !x || !r || r == x) {
        set_err("mg_residual32: bad arrays");
        return MG_ERR_ARG;
    }
    if (level == 0 && ctx->split0) {
        // the caller's arrays are in natural order: through the solver's
        // own parity-split finest FP32 buffers
        const Dims &d = ctx->L[0];
        const size_t plane = (size_t)d.ny * d.nx;
        CK(split_columns(d, x, ctx->x32[0], true, ctx->st));
        CK(split_columns(d, b, ctx->b32[0], true, ctx->st));
        CKS(residual_level<float>(ctx, 0, ctx->b32[0], ctx->x32[0], ctx->r32[0]));
        CK(split_columns(d, ctx->r32[0], r, false, ctx->st));
        for (int c = 0; c < 3; c++) {  // the solver relies on zero walls in x32[0]
            CK(cudaMemsetAsync(ctx->x32[0] + c * d.cs, 0, plane * sizeof(float), ctx->st));
            CK(cudaMemsetAsync(ctx->x32[0] + c * d.cs + d.nz * plane, 0, plane * sizeof(float),
                               ctx->st));
        }
    } else {
        CKS(residual_level<float>(ctx, level, b, x, r));
    }
    CK(cudaStreamSynchronize(ctx->st));
    return MG_OK;
}

mg_status mg_residual_restrict32(mg_ctx *ctx, int level, const float *b, const float *x,
                                 float *bc) {
    CKS(level_arg(ctx, level, 1));
    if (!b || !x || !bc) {
        set_err("mg_residual_restrict32: null array");
        return MG_ERR_ARG;
    }
    float *r = ctx->r32[level];
    if (level == 0 && ctx->split0) {
        // natural-order caller arrays through the solver's parity-split buffers
        const Dims &d = ctx->L[0];
        const size_t plane = (size_t)d.ny * d.nx;
        CK(split_columns(d, x, ctx->x32[0], true, ctx->st));
        CK(split_columns(d, b, ctx->b32[0], true, ctx->st));
        CKS(residual_restrict_level<float>(ctx, 0, ctx->b32[0], ctx->x32[0], r, bc));
        for (int c = 0; c < 3; c++) {  // the solver relies on zero walls in x32[0]
            CK(cudaMemsetAsync(ctx->x32[0] + c * d.cs, 0, plane * sizeof(float), ctx->st));
            CK(cudaMemsetAsync(ctx->x32[0] + c * d.cs + d.nz * plane, 0, plane * sizeof(float),
                               ctx->st));
        }
    } else {
        CKS(residual_restrict_level<float>(ctx, level, b, x, r, bc));
    }
    CK(cudaStreamSynchronize(ctx->st));
    return MG_OK;
}

// FP32 sweeps of a component entry point
static mg_status smooth32_entry(mg_ctx *ctx, int level, const float *b, float *x, int nsweeps,
                                bool descending) {
    if (level == 0 && ctx->split0) {
        // the caller's arrays are in natural order: convert through the
        // solver's own finest FP32 buffers
        const Dims &d = ctx->L[0];
        const size_t plane = (size_t)d.ny * d.nx;
        CK(split_columns(d, x, ctx->x32[0], true, ctx->st));
        CK(split_columns(d, b, ctx->b32[0], true, ctx->st));
        CK(cudaMemcpyAsync(ctx->xs32[0], ctx->x32[0], 3 * (size_t)d.cs * sizeof(float),
                           cudaMemcpyDeviceToDevice, ctx->st));  // partner gets the walls
        CKS(smooth<float>(ctx, 0, ctx->b32[0], ctx->x32[0], nsweeps, descending));
        CK(split_columns(d, ctx->x32[0], x, false, ctx->st));
        // the solver relies on zero walls in x32[0] and its partner
        for (float *w : {ctx->x32[0], ctx->xs32[0]})
            for (int c = 0; c < 3; c++) {
                CK(cudaMemsetAsync(w + c * d.cs, 0, plane * sizeof(float), ctx->st));
                CK(cudaMemsetAsync(w + c * d.cs + d.nz * plane, 0, plane * sizeof(float),
                                   ctx->st));
            }
    } else {
        CKS(smooth<float>(ctx, level, b, x, nsweeps, descending));
    }
    if (ctx->has_sync)
        CK(cudaMemcpyAsync(ctx->herr, ctx->sync.err, sizeof(int), cudaMemcpyDeviceToHost, ctx->st));
    CK(cudaStreamSynchronize(ctx->st));
    return sync_error(ctx);
}

mg_status mg_smooth(mg_ctx *ctx, int level, const void *b, void *x, int nsweeps, int descending,
                    int precision) {
    CKS(level_arg(ctx, level, 0));
    if (!b || !x || nsweeps < 0) {
        set_err("mg_smooth: bad arguments");
        return MG_ERR_ARG;
    }
    if (precision != MG_FP64)
        return smooth32_entry(ctx, level, (const float *)b, (float *)x, nsweeps, descending != 0);
    CKS(smooth<double>(ctx, level, (const double *)b, (double *)x, nsweeps, descending != 0));
    CK(cudaStreamSynchronize(ctx->st));
    return MG_OK;
}

mg_status mg_restrict(mg_ctx *ctx, int level, const double *r, double *bc) {
    CKS(level_arg(ctx, level, 1));
    if (!r || !bc) {
        set_err("mg_restrict: null array");
        return MG_ERR_ARG;
    }
    CK(cudaMemsetAsync(bc, 0, corner_count(ctx->L[level + 1]) * sizeof(double), ctx->st));
    CK(restrict_fw(ctx->L[level], r, bc, ctx->st));
    CK(cudaStreamSynchronize(ctx->st));
    return MG_OK;
}

mg_status mg_prolong_add(mg_ctx *ctx, int level, const double *xc, double *x) {
    CKS(level_arg(ctx, level, 1));
    if (!xc || !x) {
        set_err("mg_prolong_add: null array");
        return MG_ERR_ARG;
    }
    CK(prolong_add(ctx->L[level], xc, x, ctx->st));
    CK(cudaStreamSynchronize(ctx->st));
    return MG_OK;
}

mg_status mg_vcycle(mg_ctx *ctx, const double *b, double *x) {
    CKS(check_ctx(ctx));
    if (!b || !x) {
        set_err("mg_vcycle: null array");
        return MG_ERR_ARG;
    }
    CKS(vcycle<double>(ctx, 0, b, x));
    CK(cudaStreamSynchronize(ctx->st));
    return MG_OK;
}

static mg_status step_arg(mg_ctx *ctx) {
    CKS(check_ctx(ctx));
    if (!ctx->has_stz) {
        set_err("context was set up without stz parameters");
        return MG_ERR_ARG;
    }
    return MG_OK;
}

mg_status qs_stress_predict(mg_ctx *ctx, const double *v, const double *sigma, const double *chi,
                            double dt, double *sigma_star, double *dpl, double *sbar) {
    CKS(step_arg(ctx));
    const StepParams p = step_params(ctx, dt);
    CK(stress_predict(p, v, sigma, chi, sigma_star, dpl, sbar, ctx->st));
    if (ctx->opts.flags & MG_FLAG_ADVECT_STRESS)
        CK(stress_advect(p, v, sigma, sigma_star, ctx->st));
    CK(cudaStreamSynchronize(ctx->st));
    return MG_OK;
}

mg_status qs_chi_update(mg_ctx *ctx, const double *sigma, const double *chi, const double *dpl,
                        const double *sbar, double dt, double *chi_new) {
    CKS(step_arg(ctx));
    CK(chi_update(step_params(ctx, dt), sigma, chi, dpl, sbar, chi_new, ctx->st));
    CK(cudaStreamSynchronize(ctx->st));
    return MG_OK;
}

mg_status qs_rhs(mg_ctx *ctx, const double *sigma_star, double dt, double *b) {
    CKS(check_ctx(ctx));
    CK(div_rhs(step_params(ctx, dt), sigma_star, b, ctx->st));
    CK(cudaStreamSynchronize(ctx->st));
    return MG_OK;
}

mg_status qs_stress_correct(mg_ctx *ctx, const double *v, const double *sigma_star, double dt,
                            double *sigma) {
    CKS(check_ctx(ctx));
    CK(stress_correct(step_params(ctx, dt), v, sigma_star, sigma, nullptr, nullptr, ctx->st));
    CK(cudaStreamSynchronize(ctx->st));
    return MG_OK;
}

mg_status qs_wall_fill(mg_ctx *ctx, double *v, double t) {
    CKS(check_ctx(ctx));
    if (!ctx->has_bc) {
        set_err("context was set up without bc parameters");
        return MG_ERR_ARG;
    }
    CK(wall_fill(wall_params(ctx, t), v, ctx->st));
    CK(cudaStreamSynchronize(ctx->st));
    return MG_OK;
}

// ------------------------------------------------------------ adjoint

mg_status qs_step_adjoint(mg_ctx *ctx, const qs_state *state, double dt, double tol,
                          double work_weight, double *vbar, double *sigbar, double *chibar,
                          mg_stats *stats) {
    CKS(check_ctx(ctx));
    if (!state || !state->v || !state->sigma || !state->chi || !vbar || !sigbar || !chibar ||
        !(dt > 0.0)) {
        set_err("qs_step_adjoint: null array or dt <= 0");
        return MG_ERR_ARG;
    }
    if (!ctx->has_stz) {
        set_err("qs_step_adjoint: context was set up without stz parameters");
        return MG_ERR_ARG;
    }
    if (ctx->opts.flags & MG_FLAG_ADVECT_STRESS) {
        set_err("qs_step_adjoint: reverse mode has no adjoint of the stress advection");
        return MG_ERR_ARG;
    }
    const Dims &d = ctx->L[0];
    const size_t nc = (size_t)d.nx * d.ny * d.nz, nv = corner_count(d);
    if (!ctx->adj_rhs) {
        CKS(dalloc(ctx, &ctx->adj_rhs, nv));
        CKS(dalloc(ctx, &ctx->adj_lam, nv));
        CKS(dalloc(ctx, &ctx->adj_cb, nc));
        CKS(dalloc(ctx, &ctx->adj_db, nc));
        CKS(dalloc(ctx, &ctx->adj_sbb, nc));
        CKS(dalloc(ctx, &ctx->adj_sgb, 6 * nc));
        CKS(dalloc(ctx, &ctx->adj_Lb, 9 * nc));
    }
    const StepParams p = step_params(ctx, dt);
    // the forward D^pl and sbar of this state
    CK(stress_predict(p, state->v, state->sigma, state->chi, ctx->sig_star, ctx->dpl, ctx->sbar,
                      ctx->st));
    // stress correction (Eq. 29), then the projection solve (its own transpose)
    CK(adj_correct(p, sigbar, vbar, ctx->adj_rhs, ctx->st));
    CK(cudaMemsetAsync(ctx->adj_lam, 0, nv * sizeof(double), ctx->st));
    const mg_status s = mg_solve(ctx, ctx->adj_rhs, ctx->adj_lam, tol, stats);
    if (s != MG_OK && s != MG_ERR_NOCONV) return s;
    // chi update (Eq. 26), predictor and right-hand side (Eq. 27, Eq. 30),
    // velocity gradient (Eq. 31)
    CK(adj_chi(p, state->sigma, state->chi, ctx->dpl, ctx->sbar, chibar, ctx->adj_cb,
               ctx->adj_db, ctx->adj_sbb, ctx->adj_sgb, ctx->st));
    CK(adj_predict(p, state->v, ctx->adj_lam, state->sigma, state->chi, sigbar, ctx->adj_cb,
                   ctx->adj_db, ctx->adj_sbb, ctx->adj_sgb, chibar, ctx->adj_Lb, work_weight,
                   ctx->st));
    CK(adj_grad_transpose(p, ctx->adj_Lb, vbar, ctx->st));
    CK(cudaStreamSynchronize(ctx->st));
    return s;
}

namespace {

// device copies of a state, freed when the holder goes out of scope
struct StateStore {
    std::vector<double *> bufs;
    ~StateStore() {
        for (double *b : bufs) cudaFree(b);
    }
    double *get(size_t n) {
        void *q = nullptr;
        if (cudaMalloc(&q, n * sizeof(double)) != cudaSuccess) {
            cudaGetLastError();
            return nullptr;
        }
        bufs.push_back((double *)q);
        return (double *)q;
    }
};

}  // namespace

namespace {

size_t state_doubles(const Dims &d) { return corner_count(d) + 7 * (size_t)d.nx * d.ny * d.nz; }

cudaError_t copy_state(mg_ctx *ctx, const qs_state &from, qs_state &to) {
    const Dims &d = ctx->L[0];
    const size_t nc = (size_t)d.nx * d.ny * d.nz, nv = corner_count(d);
    cudaError_t e = cudaMemcpyAsync(to.v, from.v, nv * sizeof(double), cudaMemcpyDeviceToDevice,
                                    ctx->st);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(to.sigma, from.sigma, 6 * nc * sizeof(double),
                            cudaMemcpyDeviceToDevice, ctx->st);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(to.chi, from.chi, nc * sizeof(double), cudaMemcpyDeviceToDevice,
                            ctx->st);
    to.t = from.t;
    to.step = from.step;
    return e;
}

// checkpoint c of a contiguous block of states: v, then sigma, then chi
qs_state checkpoint_view(mg_ctx *ctx, const double *base, int c) {
    const Dims &d = ctx->L[0];
    const size_t nc = (size_t)d.nx * d.ny * d.nz, nv = corner_count(d);
    double *q = const_cast<double *>(base) + (size_t)c * state_doubles(d);
    qs_state s;
    s.v = q;
    s.sigma = q + nv;
    s.chi = q + nv + 6 * nc;
    s.t = 0.0;
    s.step = 0;
    return s;
}

mg_status work_args(mg_ctx *ctx, const void *state, int nsteps, double dt, int checkpoint_every,
                    const char *who) {
    CKS(check_ctx(ctx));
    if (!state || nsteps < 1 || checkpoint_every < 1 || !(dt > 0.0)) {
        set_err("%s: null argument, nsteps < 1, checkpoint_every < 1 or dt <= 0", who);
        return MG_ERR_ARG;
    }
    if (!ctx->has_stz || !ctx->has_bc) {
        set_err("%s: context was set up without stz/bc parameters", who);
        return MG_ERR_ARG;
    }
    if (ctx->opts.flags & MG_FLAG_ADVECT_STRESS) {
        set_err("%s: reverse mode has no adjoint of the stress advection", who);
        return MG_ERR_ARG;
    }
    return MG_OK;
}

// forward steps summing the plastic work of each (D^pl and sbar of the state
// the step starts from), keeping a copy of the state every `seg` steps in
// cp (may be null)
mg_status work_forward(mg_ctx *ctx, qs_state *state, int nsteps, double dt, double tol, int seg,
                       double *cp, double *work, mg_stats *stats) {
    const Dims &d = ctx->L[0];
    const size_t nc = (size_t)d.nx * d.ny * d.nz;
    const double wscale = 2.0 * dt * ctx->h * ctx->h * ctx->h;
    double W = 0.0;
    for (int n = 0; n < nsteps; n++) {
        if (cp && n % seg == 0) {
            qs_state q = checkpoint_view(ctx, cp, n / seg);
            CK(copy_state(ctx, *state, q));
        }
        const mg_status s = qs_step(ctx, state, dt, tol, stats);
        if (s != MG_OK) return s;
        CK(dot_cells(ctx->dpl, ctx->sbar, (long)nc, ctx->partials, ctx->st));
        CK(sum_partials(ctx->partials, ctx->dsum, ctx->st));
        CK(cudaMemcpyAsync(ctx->hsum, ctx->dsum, sizeof(double), cudaMemcpyDeviceToHost,
                           ctx->st));
        CK(cudaStreamSynchronize(ctx->st));
        W += wscale * ctx->hsum[0];
    }
    *work = W;
    return MG_OK;
}

// reverse sweep over the checkpoints written by work_forward: each segment's
// states are recomputed from its checkpoint (bitwise those of the forward
// run: its time from t0 by the same sequence of additions), then the step
// adjoints run backwards through them
mg_status work_backward(mg_ctx *ctx, const double *cp, double t0, long step0, int nsteps,
                        double dt, double tol, int seg, double *chibar, mg_stats *stats) {
    const Dims &d = ctx->L[0];
    const size_t nc = (size_t)d.nx * d.ny * d.nz, nv = corner_count(d);
    const int ncp = (nsteps + seg - 1) / seg;
    StateStore store;
    std::vector<qs_state> ss(seg);
    for (int c = 0; c < seg; c++) {
        qs_state &q = ss[c];
        q.v = store.get(nv);
        q.sigma = store.get(6 * nc);
        q.chi = store.get(nc);
        if (!q.v || !q.sigma || !q.chi) {
            set_err("qs_plastic_work_backward: out of device memory for %d segment states", seg);
            return MG_ERR_OOM;
        }
    }
    double *vbar = store.get(nv), *sigbar = store.get(6 * nc);
    if (!vbar || !sigbar) {
        set_err("qs_plastic_work_backward: out of device memory");
        return MG_ERR_OOM;
    }
    // the times of the checkpoints, as the forward steps advanced them
    std::vector<double> tcp(ncp);
    double t = t0;
    for (int n = 0; n < nsteps; n++) {
        if (n % seg == 0) tcp[n / seg] = t;
        t += dt;
    }
    CK(cudaMemsetAsync(vbar, 0, nv * sizeof(double), ctx->st));
    CK(cudaMemsetAsync(sigbar, 0, 6 * nc * sizeof(double), ctx->st));
    CK(cudaMemsetAsync(chibar, 0, nc * sizeof(double), ctx->st));
    for (int c = ncp - 1; c >= 0; c--) {
        const int n0 = c * seg, n1 = n0 + seg < nsteps ? n0 + seg : nsteps;
        qs_state q = checkpoint_view(ctx, cp, c);
        q.t = tcp[c];
        q.step = step0 + n0;
        CK(copy_state(ctx, q, ss[0]));
        for (int n = n0; n + 1 < n1; n++) {
            CK(copy_state(ctx, ss[n - n0], ss[n - n0 + 1]));
            const mg_status s = qs_step(ctx, &ss[n - n0 + 1], dt, tol, nullptr);
            if (s != MG_OK) return s;
        }
        for (int n = n1 - 1; n >= n0; n--) {
            const mg_status s = qs_step_adjoint(ctx, &ss[n - n0], dt, tol, 1.0, vbar, sigbar,
                                                chibar, stats);
            if (s != MG_OK) return s;
        }
    }
    CK(cudaStreamSynchronize(ctx->st));
    return MG_OK;
}

}  // namespace

mg_status qs_plastic_work(mg_ctx *ctx, qs_state *state, int nsteps, double dt, double tol,
                          int checkpoint_every, double *checkpoints, double *work,
                          mg_stats *stats) {
    CKS(work_args(ctx, state, nsteps, dt, checkpoint_every, "qs_plastic_work"));
    if (!state->v || !state->sigma || !state->chi || !work) {
        set_err("qs_plastic_work: null array");
        return MG_ERR_ARG;
    }
    const int seg = checkpoint_every < nsteps ? checkpoint_every : nsteps;
    return work_forward(ctx, state, nsteps, dt, tol, seg, checkpoints, work, stats);
}

mg_status qs_plastic_work_backward(mg_ctx *ctx, const double *checkpoints, double t0, long step0,
                                   int nsteps, double dt, double tol, int checkpoint_every,
                                   double *chibar, mg_stats *stats) {
    CKS(work_args(ctx, checkpoints, nsteps, dt, checkpoint_every, "qs_plastic_work_backward"));
    if (!chibar) {
        set_err("qs_plastic_work_backward: null chibar");
        return MG_ERR_ARG;
    }
    const int seg = checkpoint_every < nsteps ? checkpoint_every : nsteps;
    return work_backward(ctx, checkpoints, t0, step0, nsteps, dt, tol, seg, chibar, stats);
}

mg_status qs_plastic_work_grad(mg_ctx *ctx, qs_state *state, int nsteps, double dt, double tol,
                               int checkpoint_every, double *chibar, double *work,
                               mg_stats *stats) {
    CKS(work_args(ctx, state, nsteps, dt, checkpoint_every, "qs_plastic_work_grad"));
    if (!state->v || !state->sigma || !state->chi || !chibar || !work) {
        set_err("qs_plastic_work_grad: null array");
        return MG_ERR_ARG;
    }
    const int seg = checkpoint_every < nsteps ? checkpoint_every : nsteps;
    const int ncp = (nsteps + seg - 1) / seg;
    StateStore store;
    double *cp = store.get((size_t)ncp * state_doubles(ctx->L[0]));
    if (!cp) {
        set_err("qs_plastic_work_grad: out of device memory for %d checkpoints", ncp);
        return MG_ERR_OOM;
    }
    const double t0 = state->t;
    const long step0 = state->step;
    CKS(work_forward(ctx, state, nsteps, dt, tol, seg, cp, work, stats));
    return work_backward(ctx, cp, t0, step0, nsteps, dt, tol, seg, chibar, stats);
}

// ------------------------------------------------------------ measurement

mg_status mg_profile(mg_ctx *ctx, int enable) {
    CKS(check_ctx(ctx));
    CK(cudaStreamSynchronize(ctx->st));
    CKS(prof_drain(ctx));
    if (enable && !ctx->prof_events) {
        for (int i = 0; i < kProfSlots; i++) {
            CK(cudaEventCreate(&ctx->ev[i][0]));
            CK(cudaEventCreate(&ctx->ev[i][1]));
        }
        ctx->prof_events = true;
    }
    ctx->prof_on = enable != 0;
    ctx->prof_ms = 0.0;
    ctx->prof_sweeps = ctx->prof_launches = 0;
    return MG_OK;
}

mg_status mg_profile_read(mg_ctx *ctx, double *smooth_ms, long *smooth_sweeps,
                          long *smooth_launches) {
    CKS(check_ctx(ctx));
    CK(cudaStreamSynchronize(ctx->st));
    CKS(prof_drain(ctx));
    if (smooth_ms) *smooth_ms = ctx->prof_ms;
    if (smooth_sweeps) *smooth_sweeps = ctx->prof_sweeps;
    if (smooth_launches) *smooth_launches = ctx->prof_launches;
    return MG_OK;
}

long mg_launch_count(void) { return g_launches.load(); }

}  // extern "C"

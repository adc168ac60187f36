// qsmg_impl.h -- internal declarations shared by the library's translation
// units (kernels and host orchestration).  Not part of the public ABI.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <atomic>

namespace qsmg {

// message for mg_last_error() of the calling thread
void set_last_error(const char *fmt, ...);

// kernels launched by this library (read through mg_launch_count)
extern std::atomic<long> g_launches;
inline void count_launch(long n = 1) { g_launches.fetch_add(n, std::memory_order_relaxed); }

// cell dimensions of one level; corner arrays are (3, nz+1, ny, nx)
struct Dims {
    int nx, ny, nz;
    long cs;  // component stride (nz+1)*ny*nx
};

inline Dims make_dims(int nx, int ny, int nz) {
    Dims d;
    d.nx = nx;
    d.ny = ny;
    d.nz = nz;
    d.cs = (long)(nz + 1) * ny * nx;
    return d;
}

// Finest-level operator, Eq. (30) with the collocated stencils of section
// 3.4, scaled by -h^2/(mu dt): centre d0 = (2 lam + 8 mu)/mu on the diagonal,
// face neighbour along the component's own axis -lp = -(lam+2mu)/mu, along
// the other axes -1, edge neighbours -kq * sa * sb with kq = (lam+mu)/(4 mu).
template <typename T>
struct Fine {
    T d0, lp, kq, dinv;
};

// Coarse-level operator: one constant 27-point stencil of 3x3 blocks per
// level (Galerkin product, Eq. 36).  Reflecting one axis maps the elastic
// problem onto itself with that velocity component negated, and trilinear
// interpolation commutes with the reflection, so every level keeps the
// parity structure of the finest operator and is stored by parity class:
//   A(d)_aa = cd[a][|dx| + 2|dy| + 4|dz|]       (cd[a][0]: the centre),
//   A(d)_ab = s(d_a) s(d_b) g[c][|d_c|]          (a != b, c = 3 - a - b),
// with s() the sign of an offset; A(d)_ab = 0 when d_a or d_b is 0, so the
// centre block is diagonal and dinv[a] = 1 / cd[a][0].  Set-up checks the
// table of every level against this form.  Passed to kernels by value (it
// lives in the kernel-parameter constant bank).
template <typename T>
struct Coarse {
    T cd[3][8];
    T g[3][2];
    T dinv[3];
};

// sum over the 8 in-plane offsets (dz = 0) of A(d) u(p + d) for one node:
// u(b, dx, dy) is component b of the neighbour at in-plane offset (dx, dy)
template <typename T, class U>
__host__ __device__ __forceinline__ void coarse_plane_terms(const Coarse<T> &c, const U &u,
                                                            T o[3]) {
#pragma unroll
    for (int a = 0; a < 3; a++)
        o[a] = c.cd[a][1] * (u(a, -1, 0) + u(a, 1, 0)) + c.cd[a][2] * (u(a, 0, -1) + u(a, 0, 1)) +
               c.cd[a][3] * ((u(a, -1, -1) + u(a, 1, 1)) + (u(a, 1, -1) + u(a, -1, 1)));
    // the (x, y) coupling, |dz| = 0: sum of s(dx) s(dy) u_b
    const T qy = (u(1, 1, 1) - u(1, 1, -1)) - (u(1, -1, 1) - u(1, -1, -1));
    const T qx = (u(0, 1, 1) - u(0, 1, -1)) - (u(0, -1, 1) - u(0, -1, -1));
    o[0] += c.g[2][0] * qy;
    o[1] += c.g[2][0] * qx;
}

// sum over the 18 offsets with dz = +-1 of A(d) u(p + d) for one node, from
// the sums S_b = u_b(dz = +1) + u_b(dz = -1) and differences
// D_b = u_b(+1) - u_b(-1) at the 9 in-plane positions: sd(b, dx, dy, S, D)
// fills S and D of component b at in-plane offset (dx, dy)
template <typename T, class SD>
__host__ __device__ __forceinline__ void coarse_z_terms(const Coarse<T> &c, const SD &sd,
                                                        T o[3]) {
    T S[3][3][3], D[3][3][3];  // [b][dy + 1][dx + 1]
#pragma unroll
    for (int b = 0; b < 3; b++)
#pragma unroll
        for (int dy = -1; dy <= 1; dy++)
#pragma unroll
            for (int dx = -1; dx <= 1; dx++) sd(b, dx, dy, S[b][dy + 1][dx + 1], D[b][dy + 1][dx + 1]);
    T add[3];
#pragma unroll
    for (int a = 0; a < 3; a++)
        add[a] = c.cd[a][4] * S[a][1][1] + c.cd[a][5] * (S[a][1][0] + S[a][1][2]) +
                 c.cd[a][6] * (S[a][0][1] + S[a][2][1]) +
                 c.cd[a][7] * ((S[a][0][0] + S[a][2][2]) + (S[a][0][2] + S[a][2][0]));
    // (x, y), third axis z, |dz| = 1: s(dx) s(dy) over S
    add[0] += c.g[2][1] * ((S[1][2][2] - S[1][0][2]) - (S[1][2][0] - S[1][0][0]));
    add[1] += c.g[2][1] * ((S[0][2][2] - S[0][0][2]) - (S[0][2][0] - S[0][0][0]));
    // (x, z), third axis y: s(dx) s(dz) g[1][|dy|], the dz sum giving D
    add[0] += c.g[1][0] * (D[2][1][2] - D[2][1][0]) +
              c.g[1][1] * ((D[2][0][2] - D[2][0][0]) + (D[2][2][2] - D[2][2][0]));
    add[2] += c.g[1][0] * (D[0][1][2] - D[0][1][0]) +
              c.g[1][1] * ((D[0][0][2] - D[0][0][0]) + (D[0][2][2] - D[0][2][0]));
    // (y, z), third axis x: s(dy) s(dz) g[0][|dx|]
    add[1] += c.g[0][0] * (D[2][2][1] - D[2][0][1]) +
              c.g[0][1] * ((D[2][2][0] - D[2][0][0]) + (D[2][2][2] - D[2][0][2]));
    add[2] += c.g[0][0] * (D[1][2][1] - D[1][0][1]) +
              c.g[0][1] * ((D[1][2][0] - D[1][0][0]) + (D[1][2][2] - D[1][0][2]));
#pragma unroll
    for (int a = 0; a < 3; a++) o[a] += add[a];
}

// fixed reduction geometry: partial sums per block, then one block adds them
// in a fixed order, so every norm is bitwise reproducible
constexpr int kRedBlocks = 1216;  // 8 x 152 SMs
constexpr int kRedThreads = 256;

// ---------------------------------------------------------------- multigrid
cudaError_t gs_colour_fine(const Dims &d, const Fine<double> &f, const double *b, double *x,
                           int colour, cudaStream_t s);
cudaError_t gs_colour_fine(const Dims &d, const Fine<float> &f, const float *b, float *x,
                           int colour, cudaStream_t s);
cudaError_t gs_colour_coarse(const Dims &d, const Coarse<double> &c, const double *b, double *x,
                             int colour, cudaStream_t s);
cudaError_t gs_colour_coarse(const Dims &d, const Coarse<float> &c, const float *b, float *x,
                             int colour, cudaStream_t s);

// one-time kernel attribute set-up of the sweeps (call before any capture):
// smoother_init for the row-strip kernels, plane_init for the whole-plane one
cudaError_t smoother_init();
cudaError_t plane_init();
// FP32 finest-level residual with the persistent row-strip kernel;
// cudaErrorNotSupported when the grid or the arrays do not suit it
cudaError_t residual_fine_rows(const Dims &d, const Fine<float> &f, const float *b,
                               const float *x, float *r, cudaStream_t s, int split);
// coarse-level FP32 sweep with the persistent row-strip kernel (27-point
// block stencil); cudaErrorNotSupported when it does not apply.
// coarse_rows_fit: whether a level of these dimensions takes it.
bool coarse_rows_fit(const Dims &d);
cudaError_t gs_sweep_coarse_rows(const Dims &d, const Coarse<float> &c, const float *b,
                                 const float *vin, float *vout, bool descending, cudaStream_t s);
// Cross-CTA state of the fused finest-level sweep (device memory, zeroed at
// allocation, owned by the context): per-tile ready flags that hold the
// launch count + 1 once the tile is stored, the launch count, the CTAs done
// in the current launch, and an error word set when a bounded wait gives up.
struct SweepSync {
    int *aflag;  // [row strips][nz / 2 + 1]
    int *epoch, *done, *err;
};
// whether the fused sweep takes this grid, and the length of its flag array
bool fused_sweep_sizes(const Dims &d, long &naflag);
// FP32 finest-level sweep vin -> vout with the row-strip kernels: the fused
// one-launch sweep when sync is given and the grid suits it, else the two
// phase launches; cudaErrorNotSupported when the rows are too long for them
cudaError_t gs_sweep_fine_rows(const Dims &d, const Fine<float> &f, const float *b,
                               const float *vin, float *vout, bool descending, cudaStream_t s,
                               int split, const SweepSync *sync = nullptr);
// tiled FP32 finest-level sweep vin -> vout (two phase launches); split:
// the arrays are in parity-split column order
cudaError_t gs_sweep_fine_tiled(const Dims &d, const Fine<float> &f, const float *b,
                                const float *vin, float *vout, bool descending, cudaStream_t s,
                                int split = 0, const SweepSync *sync = nullptr);

// tiled FP32 coarse-level sweep vin -> vout (27-point block stencil)
cudaError_t gs_sweep_coarse_tiled(const Dims &d, const Coarse<float> &c, const float *b,
                                  const float *vin, float *vout, bool descending, cudaStream_t s);

// r = b - A x (interior), r walls zero
cudaError_t residual_fine(const Dims &d, const Fine<double> &f, const double *b, const double *x,
                          double *r, cudaStream_t s);
cudaError_t residual_fine(const Dims &d, const Fine<float> &f, const float *b, const float *x,
                          float *r, cudaStream_t s, int split = 0);
cudaError_t residual_coarse(const Dims &d, const Coarse<double> &c, const double *b,
                            const double *x, double *r, cudaStream_t s);
cudaError_t residual_coarse(const Dims &d, const Coarse<float> &c, const float *b, const float *x,
                            float *r, cudaStream_t s);

// FP64 fine residual with the sum of squares into partials[kRedBlocks];
// wall_only treats interior x as zero (lifted right-hand side);
// r32 (optional) receives float(r * out_scale), in parity-split column order
// if split32
cudaError_t residual_norm_fine64(const Dims &d, const Fine<double> &f, const double *b,
                                 const double *x, bool wall_only, float *r32, double out_scale,
                                 double *partials, cudaStream_t s, int split32 = 0);
// sum of squares of a level vector's interior into partials
cudaError_t sumsq(const Dims &d, const double *r, double *partials, cudaStream_t s);
// out[0] = sum of partials[0..kRedBlocks)
cudaError_t sum_partials(const double *partials, double *out, cudaStream_t s);

cudaError_t restrict_fw(const Dims &fine, const double *r, double *bc, cudaStream_t s);
// z part of the full weighting over the x-y partial sums [c][k][J][I] of
// every fine plane (component stride (nz+1) ny/2 nx/2)
cudaError_t restrict_z(const Dims &fine, const float *part, float *bc, cudaStream_t s);
// fused finest FP32 residual + restriction (row strips), or cudaErrorNotSupported
cudaError_t residual_restrict_fine_rows(const Dims &d, const Fine<float> &f, const float *b,
                                        const float *x, float *part, float *bc, cudaStream_t s,
                                        int split);
cudaError_t restrict_fw(const Dims &fine, const float *r, float *bc, cudaStream_t s,
                        int split = 0);
cudaError_t prolong_add(const Dims &fine, const double *xc, double *x, cudaStream_t s);
cudaError_t prolong_add(const Dims &fine, const float *xc, float *x, cudaStream_t s,
                        int split = 0);

// x += Ainv r on the coarsest level (dense FP64 inverse, n unknowns)
cudaError_t coarse_solve(const Dims &d, const double *Ainv, int n, const double *r, double *x,
                         cudaStream_t s);
cudaError_t coarse_solve(const Dims &d, const double *Ainv, int n, const float *r, float *x,
                         cudaStream_t s);

cudaError_t zero_interior(const Dims &d, double *x, cudaStream_t s);
// v += scale * e (interior; e in parity-split column order if split)
cudaError_t axpy_f32(const Dims &d, double scale, const float *e, double *v, cudaStream_t s,
                     int split = 0);
// corner array between natural and parity-split column order (even rows:
// x = 0, 2, ..., nx-2, then 1, 3, ..., nx-1); nx must be even
cudaError_t split_columns(const Dims &d, const float *src, float *dst, bool to_split,
                          cudaStream_t s);

// ---------------------------------------------------------------- step
struct StepParams {
    int nx, ny, nz;
    double h, dt, lam, mu;
    double tau0, eps0, c0, Delta_K, Omega, T, chi_inf, ez_K, sY, l, kB;
};
struct WallParams {
    int nx, ny, nz, kind;
    double h, t, U_B, t_ramp, omega, R, lambda_w;
};

cudaError_t stress_predict(const StepParams &p, const double *v, const double *sig,
                           const double *chi, double *sig_star, double *dpl, double *sbar,
                           cudaStream_t s);
cudaError_t chi_update(const StepParams &p, const double *sig, const double *chi,
                       const double *dpl, const double *sbar, double *chi_new, cudaStream_t s);
cudaError_t div_rhs(const StepParams &p, const double *sig_star, double *b, cudaStream_t s);
// sigma = sigma* + dt C:D(v); if chi_src is given also chi_dst = chi_src
cudaError_t stress_correct(const StepParams &p, const double *v, const double *sig_star,
                           double *sig, const double *chi_src, double *chi_dst, cudaStream_t s);
// sigma* -= dt (u.grad) sigma (ENO, Eq. 33; u the mean corner velocity of v)
cudaError_t stress_advect(const StepParams &p, const double *v, const double *sig,
                          double *sig_star, cudaStream_t s);
// Eq. (29) of one step fused with Eq. (27) of the next (same v): sig_star is
// sigma* of the finished step on entry, of the next step on return
cudaError_t correct_predict(const StepParams &p, const double *v, double *sig_star, double *sig,
                            const double *chi_src, double *chi_dst, double *dpl, double *sbar,
                            cudaStream_t s);
cudaError_t wall_fill(const WallParams &w, double *v, cudaStream_t s);
// explicit method (section 3.2), one forward-Euler step from the state
// (v, sig, chi): the stress of Eq. (25) into sig_new with D^pl and sbar of
// the state, and the velocity of Eq. (24) at the interior corners into v_new
// (rho the density, kappa the damping diffusivity)
cudaError_t explicit_stress(const StepParams &p, const double *v, const double *sig,
                            const double *chi, double *sig_new, double *dpl, double *sbar,
                            cudaStream_t s);
cudaError_t explicit_velocity(const StepParams &p, double rho, double kappa, const double *v,
                              const double *sig, double *v_new, cudaStream_t s);

// ---------------------------------------------------------------- adjoint
// (transposes of the step's equations; stored stress adjoints, see
// step_kernels.cu)
// rhs_out (interior corners) = vb1 - dt G^T (C : sigbar1); walls zero
cudaError_t adj_correct(const StepParams &p, const double *sb1, const double *vb1,
                        double *rhs_out, cudaStream_t s);
// transpose of the chi update: chib, Db, sbb per cell, sgb 6 per cell
cudaError_t adj_chi(const StepParams &p, const double *sig, const double *chi, const double *dpl,
                    const double *sbar, const double *cb1, double *chib, double *Db, double *sbb,
                    double *sgb, cudaStream_t s);
// transpose of the predictor and right-hand side: sb1 in, sigma^n adjoint
// out (in place); chib_out; Lb = velocity-gradient adjoint, 9 per cell
cudaError_t adj_predict(const StepParams &p, const double *v, const double *lam,
                        const double *sig, const double *chi, double *sb1, const double *chib,
                        const double *Db, const double *sbb, const double *sgb, double *chib_out,
                        double *Lb, double w_work, cudaStream_t s);
// vb (interior corners) = G^T Lb; walls zero
cudaError_t adj_grad_transpose(const StepParams &p, const double *Lb, double *vb,
                               cudaStream_t s);
// sum over n cells of a * b into partials[kRedBlocks]
cudaError_t dot_cells(const double *a, const double *b, long n, double *partials,
                      cudaStream_t s);

}  // namespace qsmg

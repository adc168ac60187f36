// step_kernels.cu -- pointwise kernels of the quasi-static projection step
// (section 3.3): stress predictor with the STZ rate, effective temperature,
// right-hand side of the projection system, stress correction (alone, or
// fused with the next step's predictor), wall fill, and the optional stress
// advection; the explicit method of section 3.2 (ENO advection, Eq. 33); and
// the adjoint kernels of the reverse mode.
//
// Cell arrays (nz, ny, nx); stress (6, nz, ny, nx) in the order xx, yy, zz,
// yz, xz, xy; corner arrays (3, nz+1, ny, nx).  x and y are periodic.
#include "qsmg_impl.h"

namespace qsmg {
namespace {

// 32 x 8 threads over (i, j), grid.z over planes: no flat-index division
constexpr int BX = 32, BY = 8;
const dim3 kBlock(BX, BY);
inline dim3 cell_grid(int nx, int ny, int nplanes) {
    return dim3((nx + BX - 1) / BX, (ny + BY - 1) / BY, nplanes);
}

__device__ __forceinline__ bool cell_ijk(int nx, int ny, int &i, int &j, int &k) {
    i = blockIdx.x * BX + threadIdx.x;
    j = blockIdx.y * BY + threadIdx.y;
    k = blockIdx.z;
    return i < nx && j < ny;
}

struct StzConst {
    double half_eDT_over_tau0;  // exp(-Delta/(kB T)) / (2 tau0)
    double beta;                // Omega eps0 / (kB T)
    double sY, ez_K;
};

__host__ StzConst stz_const(const StepParams &p) {
    StzConst c;
    c.half_eDT_over_tau0 = 0.5 * exp(-p.Delta_K / p.T) / p.tau0;
    c.beta = p.Omega * p.eps0 / (p.kB * p.T);
    c.sY = p.sY;
    c.ez_K = p.ez_K;
    return c;
}

// athermal STZ rate magnitude, Eqs. (20)-(22):
//   D = exp(-e_z/(kB chi)) exp(-Delta/(kB T)) cosh(Omega eps0 sbar/(kB T)) (1 - s_Y/sbar) / tau0,
// 0 at or below yield (or for chi <= 0).  FP64 is slow on this part, so the
// product exp(-e_z/chi) cosh(beta sbar) is taken as
// (exp(beta sbar - e_z/chi) + exp(-beta sbar - e_z/chi)) / 2 (two exponentials,
// no reciprocal) and 1/sbar is computed once by the caller.
__device__ __forceinline__ double stz_rate(const StzConst &c, double sbar, double inv_sbar,
                                           double chi) {
    if (!(sbar > c.sY) || !(chi > 0.0)) return 0.0;
    const double y = -c.ez_K / chi, x = c.beta * sbar;
    return (exp(x + y) + exp(y - x)) * c.half_eDT_over_tau0 * (1.0 - c.sY * inv_sbar);
}

// sbar with sbar^2 = 1/2 sigma0 : sigma0
__device__ __forceinline__ double sbar_of(const double s[6]) {
    const double m = (s[0] + s[1] + s[2]) * (1.0 / 3.0);
    const double d0 = s[0] - m, d1 = s[1] - m, d2 = s[2] - m;
    const double q = d0 * d0 + d1 * d1 + d2 * d2 + 2.0 * (s[3] * s[3] + s[4] * s[4] + s[5] * s[5]);
    return sqrt(0.5 * q);
}

// Eq. (31): G[a][b] = d v_a / d x_b at the centre of cell (i, j, k), from its
// 8 corners; each derivative averages the 4 edge differences along its axis.
// Computed for a column of cells marching up in z: each corner plane's
// contributions -- x-differences, y-differences and the sum over the 2 x 2
// corners around the column -- are formed once and shared by the cells
// below and above the plane (45 FP64 operations a cell instead of 72).
constexpr int kCellChunk = 16;  // cells of one column per thread

struct GradPlane {
    double X[3], Y[3], Z[3];
};

__device__ __forceinline__ GradPlane grad_plane(const double *__restrict__ v, long cs, long off,
                                                long r0, long r1, int i, int i1) {
    GradPlane P;
#pragma unroll
    for (int a = 0; a < 3; a++) {
        const double *g = v + a * cs + off;
        const double c00 = g[r0 + i], c10 = g[r0 + i1], c01 = g[r1 + i], c11 = g[r1 + i1];
        P.X[a] = (c10 - c00) + (c11 - c01);
        P.Y[a] = (c01 - c00) + (c11 - c10);
        P.Z[a] = (c00 + c10) + (c01 + c11);
    }
    return P;
}

// gradient of the cell between corner planes lo (k) and hi (k+1)
__device__ __forceinline__ void grad_cell(const GradPlane &lo, const GradPlane &hi, double inv4h,
                                          double G[3][3]) {
#pragma unroll
    for (int a = 0; a < 3; a++) {
        G[a][0] = (lo.X[a] + hi.X[a]) * inv4h;
        G[a][1] = (lo.Y[a] + hi.Y[a]) * inv4h;
        G[a][2] = (hi.Z[a] - lo.Z[a]) * inv4h;
    }
}

// column (i, j) of a chunk of kCellChunk cells; false if outside the grid
struct CellColumn {
    int i, j, i1, k0, k1;
    long pl, cs, r0, r1;
};
__device__ __forceinline__ bool cell_column(int nx, int ny, int nz, CellColumn &C) {
    C.i = blockIdx.x * BX + threadIdx.x;
    C.j = blockIdx.y * BY + threadIdx.y;
    if (C.i >= nx || C.j >= ny) return false;
    C.i1 = C.i + 1 < nx ? C.i + 1 : 0;
    const int j1 = C.j + 1 < ny ? C.j + 1 : 0;
    C.k0 = blockIdx.z * kCellChunk;
    C.k1 = C.k0 + kCellChunk < nz ? C.k0 + kCellChunk : nz;
    C.pl = (long)nx * ny;
    C.cs = (long)(nz + 1) * C.pl;
    C.r0 = (long)C.j * nx;
    C.r1 = (long)j1 * nx;
    return true;
}

// Eq. (27) at cell q: sigma* = sigma + dt (L sigma + sigma L^T - tr(L) sigma
// - 2 mu D^pl sigma0 / sbar) from the cell-centre gradient G of v^n and the
// cell's sigma^n (s6) and chi^n; also stores D^pl and sbar
__device__ __forceinline__ void predict_cell(const StepParams &p, const StzConst &c,
                                             const double (&G)[3][3], const double (&s6)[6],
                                             double chi_q, long q, long nc,
                                             double *__restrict__ sig_star,
                                             double *__restrict__ dpl,
                                             double *__restrict__ sbar_out) {
    // full symmetric matrix
    const double S[3][3] = {{s6[0], s6[5], s6[4]}, {s6[5], s6[1], s6[3]}, {s6[4], s6[3], s6[2]}};
    const double sb = sbar_of(s6);
    const double inv_sb = sb > 0.0 ? 1.0 / sb : 0.0;
    const double D = stz_rate(c, sb, inv_sb, chi_q);
    const double trL = G[0][0] + G[1][1] + G[2][2];
    const double m = (s6[0] + s6[1] + s6[2]) * (1.0 / 3.0);
    const double pl = (D > 0.0) ? 2.0 * p.mu * D * inv_sb : 0.0;
    // (a, b) pairs of the 6 stored components
    const int ia[6] = {0, 1, 2, 1, 0, 0}, ib[6] = {0, 1, 2, 2, 2, 1};
#pragma unroll
    for (int n = 0; n < 6; n++) {
        const int a = ia[n], b = ib[n];
        double rate = -trL * S[a][b];
#pragma unroll
        for (int e = 0; e < 3; e++) rate += G[a][e] * S[e][b] + S[a][e] * G[b][e];
        rate -= pl * (S[a][b] - (a == b ? m : 0.0));
        sig_star[n * nc + q] = S[a][b] + p.dt * rate;
    }
    dpl[q] = D;
    sbar_out[q] = sb;
}

// Eq. (29) at one cell: sigma = sigma* + dt (lam tr(D) I + 2 mu D), D = sym G
__device__ __forceinline__ void correct_cell(const StepParams &p, const double (&G)[3][3],
                                             const double (&ss)[6], double (&s6)[6]) {
    const double tr = G[0][0] + G[1][1] + G[2][2];
    const double dt = p.dt, lam = p.lam, mu = p.mu;
    s6[0] = ss[0] + dt * (lam * tr + 2.0 * mu * G[0][0]);
    s6[1] = ss[1] + dt * (lam * tr + 2.0 * mu * G[1][1]);
    s6[2] = ss[2] + dt * (lam * tr + 2.0 * mu * G[2][2]);
    s6[3] = ss[3] + dt * mu * (G[1][2] + G[2][1]);
    s6[4] = ss[4] + dt * mu * (G[0][2] + G[2][0]);
    s6[5] = ss[5] + dt * mu * (G[0][1] + G[1][0]);
}

// Eq. (27) over a column chunk of cells
__global__ void k_stress_predict(StepParams p, StzConst c, const double *__restrict__ v,
                                 const double *__restrict__ sig, const double *__restrict__ chi,
                                 double *__restrict__ sig_star, double *__restrict__ dpl,
                                 double *__restrict__ sbar_out, long nc) {
    CellColumn C;
    if (!cell_column(p.nx, p.ny, p.nz, C)) return;
    GradPlane lo = grad_plane(v, C.cs, C.k0 * C.pl, C.r0, C.r1, C.i, C.i1);
    for (int k = C.k0; k < C.k1; k++) {
        const GradPlane hi = grad_plane(v, C.cs, (k + 1) * C.pl, C.r0, C.r1, C.i, C.i1);
        const long q = k * C.pl + C.r0 + C.i;
        double G[3][3];
        grad_cell(lo, hi, 0.25 / p.h, G);
        lo = hi;
        double s6[6];
#pragma unroll
        for (int a = 0; a < 6; a++) s6[a] = sig[a * nc + q];
        predict_cell(p, c, G, s6, chi[q], q, nc, sig_star, dpl, sbar_out);
    }
}

// Eq. (26): chi' = chi + (dt/c0)[ (2 D sbar / s_Y)(chi_inf - chi) + l^2 div(D grad chi) ]
// diffusion: sum over the 6 faces of (D_P + D_N)/2 (chi_N - chi_P) / h^2;
// z ghost cells carry linearly extrapolated sigma and chi, and their D is
// the STZ rate of those extrapolated values
__global__ void k_chi_update(StepParams p, StzConst c, const double *__restrict__ sig,
                             const double *__restrict__ chi, const double *__restrict__ dpl,
                             const double *__restrict__ sbar, double *__restrict__ chi_new,
                             long nc) {
    const int nx = p.nx, ny = p.ny, nz = p.nz;
    int i, j, k;
    if (!cell_ijk(nx, ny, i, j, k)) return;
    const long q = ((long)k * ny + j) * nx + i;
    const long pl = (long)nx * ny;
    const int ip = (i + 1 < nx) ? i + 1 : 0, im = i ? i - 1 : nx - 1;
    const int jp = (j + 1 < ny) ? j + 1 : 0, jm = j ? j - 1 : ny - 1;
    const long base = (long)k * pl + (long)j * nx;
    const double c0 = chi[q], D0 = dpl[q];
    double acc = 0.0;
    long nb[4] = {base + ip, base + im, (long)k * pl + (long)jp * nx + i,
                  (long)k * pl + (long)jm * nx + i};
#pragma unroll
    for (int n = 0; n < 4; n++) acc += 0.5 * (D0 + dpl[nb[n]]) * (chi[nb[n]] - c0);
    // z neighbours, with ghosts at the walls
#pragma unroll
    for (int side = 0; side < 2; side++) {
        const int kn = side ? k + 1 : k - 1;
        double cn, Dn;
        if (kn >= 0 && kn < nz) {
            cn = chi[q + (side ? pl : -pl)];
            Dn = dpl[q + (side ? pl : -pl)];
        } else {
            // ghost: 2 * (this layer) - (next layer inward)
            const long q1 = q + (side ? -pl : pl);
            double s6[6];
#pragma unroll
            for (int a = 0; a < 6; a++) s6[a] = 2.0 * sig[a * nc + q] - sig[a * nc + q1];
            cn = 2.0 * c0 - chi[q1];
            const double sbn = sbar_of(s6);
            Dn = stz_rate(c, sbn, sbn > 0.0 ? 1.0 / sbn : 0.0, cn);
        }
        acc += 0.5 * (D0 + Dn) * (cn - c0);
    }
    const double growth = 2.0 * D0 * sbar[q] / p.sY * (p.chi_inf - c0);
    chi_new[q] = c0 + p.dt / p.c0 * (growth + (p.l * p.l) / (p.h * p.h) * acc);
}

// b = (h^2/(mu dt)) div sigma* at interior corners; the corner derivative is
// Eq. (31) shifted by half a cell: cells (i-1..i, j-1..j, k-1..k)
// corner divergence, marching up one (i, j) corner column over kDivChunk
// corner planes: each cell layer's contributions -- x-differences of
// sigma_a0, y-differences of sigma_a1 and the layer sum of sigma_a2 over the
// 2 x 2 cells around the column -- are formed once and shared by the corners
// below and above the layer (FP64 is add-bound here: about 42 adds a corner
// instead of 72)
constexpr int kDivChunk = 16;

struct DivLayer {
    double X[3], Y[3], Z[3];
};

__device__ __forceinline__ DivLayer div_layer(const double *__restrict__ ss, long nc, long base,
                                              long rj0, long rj1, int im, int i) {
    // stored component of sigma_ab: xx, yy, zz, yz, xz, xy
    const int comp[3][3] = {{0, 5, 4}, {5, 1, 3}, {4, 3, 2}};
    DivLayer L;
#pragma unroll
    for (int a = 0; a < 3; a++) {
        const double *fx = ss + comp[a][0] * nc + base, *fy = ss + comp[a][1] * nc + base,
                     *fz = ss + comp[a][2] * nc + base;
        L.X[a] = (fx[rj0 + i] - fx[rj0 + im]) + (fx[rj1 + i] - fx[rj1 + im]);
        L.Y[a] = (fy[rj1 + im] - fy[rj0 + im]) + (fy[rj1 + i] - fy[rj0 + i]);
        L.Z[a] = (fz[rj0 + im] + fz[rj0 + i]) + (fz[rj1 + im] + fz[rj1 + i]);
    }
    return L;
}

__global__ void k_div_rhs(StepParams p, const double *__restrict__ ss, double *__restrict__ b,
                          double scale) {
    const int nx = p.nx, ny = p.ny, nz = p.nz;
    const int i = blockIdx.x * BX + threadIdx.x, j = blockIdx.y * BY + threadIdx.y;
    if (i >= nx || j >= ny) return;
    const int k0 = 1 + blockIdx.z * kDivChunk;
    const int k1 = k0 + kDivChunk < nz ? k0 + kDivChunk : nz;  // corners k0 .. k1-1
    const int im = i ? i - 1 : nx - 1, jm = j ? j - 1 : ny - 1;
    const long nc = (long)nx * ny * nz, pl = (long)nx * ny;
    const long rj0 = (long)jm * nx, rj1 = (long)j * nx;
    const long cs = (long)(nz + 1) * pl;
    DivLayer lo = div_layer(ss, nc, (long)(k0 - 1) * pl, rj0, rj1, im, i);
    for (int k = k0; k < k1; k++) {
        const DivLayer hi = div_layer(ss, nc, (long)k * pl, rj0, rj1, im, i);
        const long node = (long)k * pl + (long)j * nx + i;
#pragma unroll
        for (int a = 0; a < 3; a++)
            b[a * cs + node] = scale * ((lo.X[a] + hi.X[a]) + (lo.Y[a] + hi.Y[a]) + (hi.Z[a] - lo.Z[a]));
        lo = hi;
    }
}

// Eq. (29) over a column chunk of cells; chi_dst <- chi_src on the way
// (the step's new chi, when chi_dst is not null)
__global__ void k_stress_correct(StepParams p, const double *__restrict__ v,
                                 const double *__restrict__ ss, double *__restrict__ sig,
                                 const double *__restrict__ chi_src, double *__restrict__ chi_dst,
                                 long nc) {
    CellColumn C;
    if (!cell_column(p.nx, p.ny, p.nz, C)) return;
    GradPlane lo = grad_plane(v, C.cs, C.k0 * C.pl, C.r0, C.r1, C.i, C.i1);
    for (int k = C.k0; k < C.k1; k++) {
        const GradPlane hi = grad_plane(v, C.cs, (k + 1) * C.pl, C.r0, C.r1, C.i, C.i1);
        const long q = k * C.pl + C.r0 + C.i;
        double G[3][3];
        grad_cell(lo, hi, 0.25 / p.h, G);
        lo = hi;
        double s6[6], ss6[6];
#pragma unroll
        for (int a = 0; a < 6; a++) ss6[a] = ss[a * nc + q];
        correct_cell(p, G, ss6, s6);
#pragma unroll
        for (int a = 0; a < 6; a++) sig[a * nc + q] = s6[a];
        if (chi_dst) chi_dst[q] = chi_src[q];
    }
}

// Eq. (29) of step n and Eq. (27) of step n+1 in one pass: both use the
// gradient of the same velocity v^{n+1}, so it is formed once, and sigma^{n+1}
// goes from the correction straight into the predictor without a round trip
// through memory.  sig_star holds sigma* of step n on entry and of step n+1
// on return (each cell reads and writes only its own entries); sig receives
// sigma^{n+1}, chi_dst the step's new chi (chi_src).
__global__ void k_correct_predict(StepParams p, StzConst c, const double *__restrict__ v,
                                  double *__restrict__ sig_star, double *__restrict__ sig,
                                  const double *__restrict__ chi_src,
                                  double *__restrict__ chi_dst, double *__restrict__ dpl,
                                  double *__restrict__ sbar_out, long nc) {
    CellColumn C;
    if (!cell_column(p.nx, p.ny, p.nz, C)) return;
    GradPlane lo = grad_plane(v, C.cs, C.k0 * C.pl, C.r0, C.r1, C.i, C.i1);
    for (int k = C.k0; k < C.k1; k++) {
        const GradPlane hi = grad_plane(v, C.cs, (k + 1) * C.pl, C.r0, C.r1, C.i, C.i1);
        const long q = k * C.pl + C.r0 + C.i;
        double G[3][3];
        grad_cell(lo, hi, 0.25 / p.h, G);
        lo = hi;
        double s6[6], ss6[6];
#pragma unroll
        for (int a = 0; a < 6; a++) ss6[a] = sig_star[a * nc + q];
        correct_cell(p, G, ss6, s6);
#pragma unroll
        for (int a = 0; a < 6; a++) sig[a * nc + q] = s6[a];
        const double chi_q = chi_src[q];
        chi_dst[q] = chi_q;
        predict_cell(p, c, G, s6, chi_q, q, nc, sig_star, dpl, sbar_out);
    }
}

// wall velocities of section 4 (simple shear with ramp) and section 5 (disc)
__global__ void k_wall_fill(WallParams w, double *__restrict__ v) {
    const int i = blockIdx.x * BX + threadIdx.x, j = blockIdx.y * BY + threadIdx.y;
    if (i >= w.nx || j >= w.ny) return;
    const long pl = (long)w.nx * w.ny;
    const long t = (long)j * w.nx + i;
    double top[3] = {0.0, 0.0, 0.0}, bot[3] = {0.0, 0.0, 0.0};
    if (w.kind == 0) {
        const double U = (w.t < w.t_ramp) ? w.U_B * w.t / w.t_ramp : w.U_B;
        top[0] = U;
        bot[0] = -U;
    } else {
        const double L = 0.5 * w.nx * w.h;
        const double x = -L + i * w.h, y = -0.5 * w.ny * w.h + j * w.h;
        const double r2 = (x * x + y * y) / (L * L), R2 = w.R * w.R;
        const double f = (r2 < R2) ? 1.0 : exp(-w.lambda_w * (r2 - R2) * (r2 - R2));
        top[0] = -w.omega * y * f;
        top[1] = w.omega * x * f;
        const double sgn = (w.kind == 2) ? 1.0 : (w.kind == 3 ? -1.0 : 0.0);
        bot[0] = sgn * top[0];
        bot[1] = sgn * top[1];
    }
    const long cs = (long)(w.nz + 1) * pl;
#pragma unroll
    for (int a = 0; a < 3; a++) {
        v[a * cs + t] = bot[a];
        v[a * cs + (long)w.nz * pl + t] = top[a];
    }
}

// ------------------------------------------------------------ explicit method
// (section 3.2): forward Euler of Eqs. (24)-(26) with ENO advection (Eq. 33)

// ENO first derivative, Eq. (33), from the values at offsets -2..2 along one
// axis and the velocity component u along it: the one-sided three-point
// stencil on the upwind side where that side is smoother than the centre,
// else the centred difference.  The smoothness test compares the magnitudes
// of the undivided second differences: the curvatures of Eq. (33) are those
// divided by the same h^2 > 0, which cannot reorder them (the division is
// monotone), and FP64 division is costly here; inv2h = 1 / (2h).
__device__ __forceinline__ double eno_d(double fm2, double fm1, double f0, double fp1, double fp2,
                                        double u, double inv2h) {
    const double cm = fabs(f0 - 2.0 * fm1 + fm2);
    const double c0 = fabs(fp1 - 2.0 * f0 + fm1);
    const double cp = fabs(fp2 - 2.0 * fp1 + f0);
    if (u < 0.0 && c0 > cp) return (-fp2 + 4.0 * fp1 - 3.0 * f0) * inv2h;
    if (u > 0.0 && c0 > cm) return (3.0 * f0 - 4.0 * fm1 + fm2) * inv2h;
    return (fp1 - fm1) * inv2h;
}

// (u.grad) sigma_n at cell (i, j, k) for the 6 stored components: ENO
// derivatives (Eq. 33) along x and y (wrapping) and z, where cell fields two
// layers beyond the z boundaries are extrapolated linearly from the two
// layers next to them; u is the cell's advecting velocity
__device__ __forceinline__ void stress_advection(const StepParams &p,
                                                 const double *__restrict__ sig, long nc, int i,
                                                 int j, int k, const double (&u)[3],
                                                 double inv2h, double (&adv)[6]) {
    const int nx = p.nx, ny = p.ny, nz = p.nz;
    const long pl = (long)nx * ny;
    int ix[5], jy[5];
#pragma unroll
    for (int m = 0; m < 5; m++) {
        int a = i + m - 2, b = j + m - 2;
        ix[m] = a < 0 ? a + nx : (a >= nx ? a - nx : a);
        jy[m] = b < 0 ? b + ny : (b >= ny ? b - ny : b);
    }
#pragma unroll
    for (int n = 0; n < 6; n++) {
        const double *f = sig + n * nc;
        double fx[5], fy[5], fz[5];
#pragma unroll
        for (int m = 0; m < 5; m++) {
            fx[m] = f[(long)k * pl + (long)j * nx + ix[m]];
            fy[m] = f[(long)k * pl + (long)jy[m] * nx + i];
            const int kk = k + m - 2;
            const long col = (long)j * nx + i;
            if (kk < 0)
                fz[m] = f[col] + kk * (f[pl + col] - f[col]);
            else if (kk > nz - 1)
                fz[m] = f[(long)(nz - 1) * pl + col] +
                        (kk - (nz - 1)) * (f[(long)(nz - 1) * pl + col] - f[(long)(nz - 2) * pl + col]);
            else
                fz[m] = f[(long)kk * pl + col];
        }
        adv[n] = u[0] * eno_d(fx[0], fx[1], fx[2], fx[3], fx[4], u[0], inv2h) +
                 u[1] * eno_d(fy[0], fy[1], fy[2], fy[3], fy[4], u[1], inv2h) +
                 u[2] * eno_d(fz[0], fz[1], fz[2], fz[3], fz[4], u[2], inv2h);
    }
}

// Eq. (25) at cell centres: sigma' = sigma + dt (-(u.grad) sigma + L sigma +
// sigma L^T - tr(L) sigma + C:(D - D^pl sigma0 / sbar)), L the Eq. (31)
// gradient of v, u the mean of the cell's 8 corner velocities; the ENO
// stencils reach two cells out, z ghost cells extrapolate each component
// linearly from the two layers next to the wall; D^pl and sbar of the state
// are written for the chi update
__global__ void k_explicit_stress(StepParams p, StzConst c, const double *__restrict__ v,
                                  const double *__restrict__ sig, const double *__restrict__ chi,
                                  double *__restrict__ sig_new, double *__restrict__ dpl,
                                  double *__restrict__ sbar_out, long nc) {
    const int nx = p.nx, ny = p.ny, nz = p.nz;
    int i, j, k;
    if (!cell_ijk(nx, ny, i, j, k)) return;
    const long pl = (long)nx * ny, cs = (long)(nz + 1) * pl;
    const int i1 = i + 1 < nx ? i + 1 : 0, j1 = j + 1 < ny ? j + 1 : 0;
    const double h = p.h, inv2h = 0.5 / p.h;
    double G[3][3], u[3];
#pragma unroll
    for (int a = 0; a < 3; a++) {
        const double *g = v + a * cs;
        const long b0 = (long)k * pl, b1 = b0 + pl, r0 = (long)j * nx, r1 = (long)j1 * nx;
        const double c000 = g[b0 + r0 + i], c001 = g[b0 + r0 + i1], c010 = g[b0 + r1 + i],
                     c011 = g[b0 + r1 + i1], c100 = g[b1 + r0 + i], c101 = g[b1 + r0 + i1],
                     c110 = g[b1 + r1 + i], c111 = g[b1 + r1 + i1];
        G[a][0] = ((c001 - c000) + (c011 - c010) + (c101 - c100) + (c111 - c110)) * (0.25 / h);
        G[a][1] = ((c010 - c000) + (c011 - c001) + (c110 - c100) + (c111 - c101)) * (0.25 / h);
        G[a][2] = ((c100 - c000) + (c110 - c010) + (c101 - c001) + (c111 - c011)) * (0.25 / h);
        u[a] = 0.125 * (((c000 + c001) + (c010 + c011)) + ((c100 + c101) + (c110 + c111)));
    }
    const long q = (long)k * pl + (long)j * nx + i;
    double s6[6], adv[6];
#pragma unroll
    for (int n = 0; n < 6; n++) s6[n] = sig[n * nc + q];
    stress_advection(p, sig, nc, i, j, k, u, inv2h, adv);
    const double S[3][3] = {{s6[0], s6[5], s6[4]}, {s6[5], s6[1], s6[3]}, {s6[4], s6[3], s6[2]}};
    const double sb = sbar_of(s6);
    const double inv_sb = sb > 0.0 ? 1.0 / sb : 0.0;
    const double D = stz_rate(c, sb, inv_sb, chi[q]);
    const double trL = G[0][0] + G[1][1] + G[2][2];
    const double m3 = (s6[0] + s6[1] + s6[2]) * (1.0 / 3.0);
    const double pl_ = (D > 0.0) ? 2.0 * p.mu * D * inv_sb : 0.0;
    const int ia[6] = {0, 1, 2, 1, 0, 0}, ib[6] = {0, 1, 2, 2, 2, 1};
#pragma unroll
    for (int n = 0; n < 6; n++) {
        const int a = ia[n], b = ib[n];
        double rate = -adv[n] - trL * S[a][b];
#pragma unroll
        for (int e = 0; e < 3; e++) rate += G[a][e] * S[e][b] + S[a][e] * G[b][e];
        rate += (a == b ? p.lam * trL : 0.0) + p.mu * (G[a][b] + G[b][a]);
        rate -= pl_ * (S[a][b] - (a == b ? m3 : 0.0));
        sig_new[n * nc + q] = S[a][b] + p.dt * rate;
    }
    dpl[q] = D;
    sbar_out[q] = sb;
}

// the stress advection of the general constitutive law (section 2), which
// Eq. (27) drops, as an option of the quasi-static step: sigma* -= dt (u.grad)
// sigma^n, u the mean of the cell's 8 corner velocities of v^n (the
// explicit method's advection, Eq. 33 and its ghosts)
__global__ void k_stress_advect(StepParams p, const double *__restrict__ v,
                                const double *__restrict__ sig, double *__restrict__ sig_star,
                                long nc) {
    const int nx = p.nx, ny = p.ny, nz = p.nz;
    int i, j, k;
    if (!cell_ijk(nx, ny, i, j, k)) return;
    const long pl = (long)nx * ny, cs = (long)(nz + 1) * pl;
    const int i1 = i + 1 < nx ? i + 1 : 0, j1 = j + 1 < ny ? j + 1 : 0;
    double u[3];
#pragma unroll
    for (int a = 0; a < 3; a++) {
        const double *g = v + a * cs;
        const long b0 = (long)k * pl, b1 = b0 + pl, r0 = (long)j * nx, r1 = (long)j1 * nx;
        u[a] = 0.125 * (((g[b0 + r0 + i] + g[b0 + r0 + i1]) + (g[b0 + r1 + i] + g[b0 + r1 + i1])) +
                        ((g[b1 + r0 + i] + g[b1 + r0 + i1]) + (g[b1 + r1 + i] + g[b1 + r1 + i1])));
    }
    double adv[6], ss[6];
    stress_advection(p, sig, nc, i, j, k, u, 0.5 / p.h, adv);
    const long q = (long)k * pl + (long)j * nx + i;
#pragma unroll
    for (int n = 0; n < 6; n++) ss[n] = sig_star[n * nc + q];
#pragma unroll
    for (int n = 0; n < 6; n++) sig_star[n * nc + q] = ss[n] - p.dt * adv[n];
}

// Eq. (24) at interior corners (k = 1 .. nz-1):
//   v' = v + dt (-(v.grad) v + div sigma / rho + kappa lap v),
// the divergence the corner version of Eq. (31) over the 8 cells around the
// corner, the Laplacian Eq. (32) along each axis, ENO advection with the
// corner's own velocity; corners up to two planes beyond a wall reflect v
// through the wall value, v(-m) = 2 v(0) - v(m)
__global__ void k_explicit_velocity(StepParams p, double inv_rho, double kappa,
                                    const double *__restrict__ v, const double *__restrict__ sig,
                                    double *__restrict__ v_new, long nc) {
    const int nx = p.nx, ny = p.ny, nz = p.nz;
    const int i = blockIdx.x * BX + threadIdx.x, j = blockIdx.y * BY + threadIdx.y;
    const int k = blockIdx.z + 1;
    if (i >= nx || j >= ny) return;
    const long pl = (long)nx * ny, cs = (long)(nz + 1) * pl;
    const double h = p.h, inv_h2 = 1.0 / (p.h * p.h), inv2h = 0.5 / p.h;
    const int im = i ? i - 1 : nx - 1, jm = j ? j - 1 : ny - 1;
    const int ip = i + 1 < nx ? i + 1 : 0, jp = j + 1 < ny ? j + 1 : 0;
    const long node = (long)k * pl + (long)j * nx + i;
    int ix[5], jy[5];
#pragma unroll
    for (int m = 0; m < 5; m++) {
        int a = i + m - 2, b = j + m - 2;
        ix[m] = a < 0 ? a + nx : (a >= nx ? a - nx : a);
        jy[m] = b < 0 ? b + ny : (b >= ny ? b - ny : b);
    }
    const double u[3] = {v[node], v[cs + node], v[2 * cs + node]};
    const int comp[3][3] = {{0, 5, 4}, {5, 1, 3}, {4, 3, 2}};
    const long c0 = (long)(k - 1) * pl, c1 = (long)k * pl;
    const long rm = (long)jm * nx, r0 = (long)j * nx;
#pragma unroll
    for (int a = 0; a < 3; a++) {
        const double *fx = sig + comp[a][0] * nc, *fy = sig + comp[a][1] * nc,
                     *fz = sig + comp[a][2] * nc;
        const double div =
            (((fx[c0 + rm + i] - fx[c0 + rm + im]) + (fx[c0 + r0 + i] - fx[c0 + r0 + im])) +
             ((fx[c1 + rm + i] - fx[c1 + rm + im]) + (fx[c1 + r0 + i] - fx[c1 + r0 + im])) +
             ((fy[c0 + r0 + im] - fy[c0 + rm + im]) + (fy[c0 + r0 + i] - fy[c0 + rm + i])) +
             ((fy[c1 + r0 + im] - fy[c1 + rm + im]) + (fy[c1 + r0 + i] - fy[c1 + rm + i])) +
             ((fz[c1 + rm + im] - fz[c0 + rm + im]) + (fz[c1 + rm + i] - fz[c0 + rm + i])) +
             ((fz[c1 + r0 + im] - fz[c0 + r0 + im]) + (fz[c1 + r0 + i] - fz[c0 + r0 + i]))) *
            (0.25 / h);
        const double *g = v + a * cs;
        const double w0 = g[node];
        const double lap = ((g[node - i + ip] - 2.0 * w0 + g[node - i + im]) +
                            (g[node - (long)j * nx + (long)jp * nx] - 2.0 * w0 +
                             g[node - (long)j * nx + (long)jm * nx]) +
                            (g[node + pl] - 2.0 * w0 + g[node - pl])) *
                           inv_h2;
        double fxl[5], fyl[5], fzl[5];
#pragma unroll
        for (int m = 0; m < 5; m++) {
            fxl[m] = g[(long)k * pl + (long)j * nx + ix[m]];
            fyl[m] = g[(long)k * pl + (long)jy[m] * nx + i];
            const int kk = k + m - 2;
            const long col = (long)j * nx + i;
            if (kk < 0)
                fzl[m] = 2.0 * g[col] - g[(long)(-kk) * pl + col];
            else if (kk > nz)
                fzl[m] = 2.0 * g[(long)nz * pl + col] - g[(long)(2 * nz - kk) * pl + col];
            else
                fzl[m] = g[(long)kk * pl + col];
        }
        const double adv = u[0] * eno_d(fxl[0], fxl[1], fxl[2], fxl[3], fxl[4], u[0], inv2h) +
                           u[1] * eno_d(fyl[0], fyl[1], fyl[2], fyl[3], fyl[4], u[1], inv2h) +
                           u[2] * eno_d(fzl[0], fzl[1], fzl[2], fzl[3], fzl[4], u[2], inv2h);
        v_new[a * cs + node] = w0 + p.dt * (-adv + div * inv_rho + kappa * lap);
    }
}

}  // namespace

cudaError_t stress_predict(const StepParams &p, const double *v, const double *sig,
                           const double *chi, double *sig_star, double *dpl, double *sbar,
                           cudaStream_t s) {
    const long nc = (long)p.nx * p.ny * p.nz;
    k_stress_predict<<<cell_grid(p.nx, p.ny, (p.nz + kCellChunk - 1) / kCellChunk), kBlock, 0, s>>>(p, stz_const(p), v, sig, chi,
                                                                    sig_star, dpl, sbar, nc);
    count_launch();
    return cudaGetLastError();
}

cudaError_t chi_update(const StepParams &p, const double *sig, const double *chi,
                       const double *dpl, const double *sbar, double *chi_new, cudaStream_t s) {
    const long nc = (long)p.nx * p.ny * p.nz;
    k_chi_update<<<cell_grid(p.nx, p.ny, p.nz), kBlock, 0, s>>>(p, stz_const(p), sig, chi, dpl,
                                                                sbar, chi_new, nc);
    count_launch();
    return cudaGetLastError();
}

cudaError_t div_rhs(const StepParams &p, const double *sig_star, double *b, cudaStream_t s) {
    const long pl = (long)p.nx * p.ny;
    const double scale = p.h * p.h / (p.mu * p.dt) * (0.25 / p.h);
    cudaError_t e;
    const long cs = (long)(p.nz + 1) * pl;
    for (int a = 0; a < 3; a++) {  // wall planes of b are not part of the system
        e = cudaMemsetAsync(b + a * cs, 0, pl * sizeof(double), s);
        if (e != cudaSuccess) return e;
        e = cudaMemsetAsync(b + a * cs + (long)p.nz * pl, 0, pl * sizeof(double), s);
        if (e != cudaSuccess) return e;
    }
    k_div_rhs<<<cell_grid(p.nx, p.ny, (p.nz - 1 + kDivChunk - 1) / kDivChunk), kBlock, 0, s>>>(
        p, sig_star, b, scale);
    count_launch();
    return cudaGetLastError();
}

cudaError_t stress_correct(const StepParams &p, const double *v, const double *sig_star,
                           double *sig, const double *chi_src, double *chi_dst, cudaStream_t s) {
    const long nc = (long)p.nx * p.ny * p.nz;
    k_stress_correct<<<cell_grid(p.nx, p.ny, (p.nz + kCellChunk - 1) / kCellChunk), kBlock, 0, s>>>(p, v, sig_star, sig, chi_src,
                                                                    chi_dst, nc);
    count_launch();
    return cudaGetLastError();
}

cudaError_t stress_advect(const StepParams &p, const double *v, const double *sig,
                          double *sig_star, cudaStream_t s) {
    const long nc = (long)p.nx * p.ny * p.nz;
    k_stress_advect<<<cell_grid(p.nx, p.ny, p.nz), kBlock, 0, s>>>(p, v, sig, sig_star, nc);
    count_launch();
    return cudaGetLastError();
}

cudaError_t correct_predict(const StepParams &p, const double *v, double *sig_star, double *sig,
                            const double *chi_src, double *chi_dst, double *dpl, double *sbar,
                            cudaStream_t s) {
    const long nc = (long)p.nx * p.ny * p.nz;
    k_correct_predict<<<cell_grid(p.nx, p.ny, (p.nz + kCellChunk - 1) / kCellChunk), kBlock, 0,
                        s>>>(p, stz_const(p), v, sig_star, sig, chi_src, chi_dst, dpl, sbar, nc);
    count_launch();
    return cudaGetLastError();
}

cudaError_t wall_fill(const WallParams &w, double *v, cudaStream_t s) {
    k_wall_fill<<<cell_grid(w.nx, w.ny, 1), kBlock, 0, s>>>(w, v);
    count_launch();
    return cudaGetLastError();
}

cudaError_t explicit_stress(const StepParams &p, const double *v, const double *sig,
                            const double *chi, double *sig_new, double *dpl, double *sbar,
                            cudaStream_t s) {
    const long nc = (long)p.nx * p.ny * p.nz;
    k_explicit_stress<<<cell_grid(p.nx, p.ny, p.nz), kBlock, 0, s>>>(p, stz_const(p), v, sig, chi,
                                                                     sig_new, dpl, sbar, nc);
    count_launch();
    return cudaGetLastError();
}

cudaError_t explicit_velocity(const StepParams &p, double rho, double kappa, const double *v,
                              const double *sig, double *v_new, cudaStream_t s) {
    const long nc = (long)p.nx * p.ny * p.nz;
    if (p.nz < 2) return cudaSuccess;
    k_explicit_velocity<<<cell_grid(p.nx, p.ny, p.nz - 1), kBlock, 0, s>>>(p, 1.0 / rho, kappa, v,
                                                                          sig, v_new, nc);
    count_launch();
    return cudaGetLastError();
}

}  // namespace qsmg

// ------------------------------------------------------------------ adjoint
//
// Reverse of one projection step for the gradient of an objective through
// the step: given the adjoints (vbar, sigbar, chibar) of the state after the
// step, the adjoints of the state before it.  Each kernel is the transpose
// of one forward equation (Eqs. 26, 27, 29, 31 and the right-hand side of
// Eq. 30); the projection solve is its own transpose (the scaled operator is
// symmetric) and runs through the multigrid solver.  Stored stress adjoints
// follow the stored components: for an off-diagonal component the adjoint is
// the sum of the two full-matrix entries, so the full-matrix adjoint is half
// of it.

namespace qsmg {
namespace {

// STZ rate (as stz_rate) with its partial derivatives in sbar and chi
__device__ __forceinline__ void stz_rate_d(const StzConst &c, double sbar, double inv_sbar,
                                           double chi, double &D, double &Ds, double &Dc) {
    if (!(sbar > c.sY) || !(chi > 0.0)) {
        D = Ds = Dc = 0.0;
        return;
    }
    const double y = -c.ez_K / chi, x = c.beta * sbar;
    const double ep = exp(x + y), em = exp(y - x);
    const double f = 1.0 - c.sY * inv_sbar;
    D = (ep + em) * c.half_eDT_over_tau0 * f;
    Ds = c.half_eDT_over_tau0 * (c.beta * (ep - em) * f + (ep + em) * c.sY * inv_sbar * inv_sbar);
    Dc = D * c.ez_K / (chi * chi);
}

// deviatoric part and sbar of a stored stress
__device__ __forceinline__ void dev_of(const double s[6], double S0[3][3], double &sb,
                                       double &inv_sb) {
    const double m = (s[0] + s[1] + s[2]) * (1.0 / 3.0);
    S0[0][0] = s[0] - m;
    S0[1][1] = s[1] - m;
    S0[2][2] = s[2] - m;
    S0[1][2] = S0[2][1] = s[3];
    S0[0][2] = S0[2][0] = s[4];
    S0[0][1] = S0[1][0] = s[5];
    sb = sbar_of(s);
    inv_sb = sb > 0.0 ? 1.0 / sb : 0.0;
}

// stored adjoint of a symmetric full-matrix adjoint X (added, times w)
__device__ __forceinline__ void add_stored(double out[6], const double X[3][3], double w) {
    out[0] += w * X[0][0];
    out[1] += w * X[1][1];
    out[2] += w * X[2][2];
    out[3] += w * (X[1][2] + X[2][1]);
    out[4] += w * (X[0][2] + X[2][0]);
    out[5] += w * (X[0][1] + X[1][0]);
}

// Transpose of the chi diffusion at one z-wall ghost face.  Cell P (boundary
// layer) has a ghost neighbour with chi_g = 2 chi_P - chi_Q and sigma_g =
// 2 sigma_P - sigma_Q (Q the next layer inward); its face term in P's update
// is a (D_P + D_g)/2 (chi_g - chi_P), a = chibar'_P dt l^2 / (c0 h^2).
// Returns the adjoint contributions: to chi_P (cP), chi_Q (cQ), D_P (dP) and
// the full-matrix stress adjoint Sg of the ghost (P receives 2 Sg, Q -Sg).
struct GhostAdj {
    double cP, cQ, dP;
    double Sg[3][3];
};
__device__ __forceinline__ GhostAdj ghost_adj(const StzConst &c, const double *__restrict__ sig,
                                              const double *__restrict__ chi,
                                              const double *__restrict__ dpl, long nc, long qP,
                                              long qQ, double a) {
    GhostAdj G;
    double sg[6];
#pragma unroll
    for (int n = 0; n < 6; n++) sg[n] = 2.0 * sig[n * nc + qP] - sig[n * nc + qQ];
    const double cP = chi[qP], cg = 2.0 * cP - chi[qQ], DP = dpl[qP];
    double S0[3][3], sb, inv;
    dev_of(sg, S0, sb, inv);
    double Dg, Dgs, Dgc;
    stz_rate_d(c, sb, inv, cg, Dg, Dgs, Dgc);
    const double half_gap = 0.5 * (cg - cP);
    // d/dchi_g = a (D_P + D_g)/2 + a (chi_g - chi_P)/2 dD_g/dchi_g; chi_g = 2 chi_P - chi_Q
    const double dg = a * 0.5 * (DP + Dg) + a * half_gap * Dgc;
    G.cP = -a * 0.5 * (DP + Dg) + 2.0 * dg;
    G.cQ = -dg;
    G.dP = a * half_gap;
    const double w = a * half_gap * Dgs * 0.5 * inv;  // Dbar_g dD_g/dsbar_g / (2 sbar_g)
#pragma unroll
    for (int r = 0; r < 3; r++)
#pragma unroll
        for (int s = 0; s < 3; s++) G.Sg[r][s] = w * S0[r][s];
    return G;
}

// Transpose of Eq. (26) in gather form, per cell P: chib (adjoint of chi^n
// through the chi update), Db and sbb (adjoints of D^pl_P and sbar_P), and
// sgb (stress adjoint from the z-wall ghosts, stored; zero away from the two
// outer layers on each side)
__global__ void k_adj_chi(StepParams p, StzConst c, const double *__restrict__ sig,
                          const double *__restrict__ chi, const double *__restrict__ dpl,
                          const double *__restrict__ sbar, const double *__restrict__ cb1,
                          double *__restrict__ chib, double *__restrict__ Db,
                          double *__restrict__ sbb, double *__restrict__ sgb, long nc) {
    const int nx = p.nx, ny = p.ny, nz = p.nz;
    int i, j, k;
    if (!cell_ijk(nx, ny, i, j, k)) return;
    const long pl = (long)nx * ny;
    const long q = (long)k * pl + (long)j * nx + i;
    const double kap = p.dt / p.c0, kd = kap * (p.l * p.l) / (p.h * p.h);
    const double bP = cb1[q], cP = chi[q], DP = dpl[q], sP = sbar[q];
    double cb = bP - bP * kap * 2.0 * DP * sP / p.sY;
    double db = bP * kap * 2.0 * sP / p.sY * (p.chi_inf - cP);
    const double sbv = bP * kap * 2.0 * DP / p.sY * (p.chi_inf - cP);
    const int ip = (i + 1 < nx) ? i + 1 : 0, im = i ? i - 1 : nx - 1;
    const int jp = (j + 1 < ny) ? j + 1 : 0, jm = j ? j - 1 : ny - 1;
    long nb[6];
    int nn = 0;
    nb[nn++] = (long)k * pl + (long)j * nx + ip;
    nb[nn++] = (long)k * pl + (long)j * nx + im;
    nb[nn++] = (long)k * pl + (long)jp * nx + i;
    nb[nn++] = (long)k * pl + (long)jm * nx + i;
    if (k + 1 < nz) nb[nn++] = q + pl;
    if (k > 0) nb[nn++] = q - pl;
    for (int n = 0; n < nn; n++) {
        const double bN = cb1[nb[n]], DN = dpl[nb[n]], cN = chi[nb[n]];
        cb += kd * 0.5 * (DP + DN) * (bN - bP);
        db += kd * 0.5 * (cN - cP) * (bP - bN);
    }
    double sg[6] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
    // this cell's own ghost faces
    if (k == nz - 1) {
        const GhostAdj G = ghost_adj(c, sig, chi, dpl, nc, q, q - pl, bP * kd);
        cb += G.cP;
        db += G.dP;
        add_stored(sg, G.Sg, 2.0);
    }
    if (k == 0) {
        const GhostAdj G = ghost_adj(c, sig, chi, dpl, nc, q, q + pl, bP * kd);
        cb += G.cP;
        db += G.dP;
        add_stored(sg, G.Sg, 2.0);
    }
    // this cell as the inner layer of a neighbour's ghost
    if (k == nz - 2) {
        const GhostAdj G = ghost_adj(c, sig, chi, dpl, nc, q + pl, q, cb1[q + pl] * kd);
        cb += G.cQ;
        add_stored(sg, G.Sg, -1.0);
    }
    if (k == 1) {
        const GhostAdj G = ghost_adj(c, sig, chi, dpl, nc, q - pl, q, cb1[q - pl] * kd);
        cb += G.cQ;
        add_stored(sg, G.Sg, -1.0);
    }
    chib[q] = cb;
    Db[q] = db;
    sbb[q] = sbv;
#pragma unroll
    for (int n = 0; n < 6; n++) sgb[n * nc + q] = sg[n];
}

// Transpose of Eq. (27) (with the work term and the right-hand side of
// Eq. 30 folded in), per cell: from the stored adjoint of sigma^{n+1}
// (sb1, which is also that of sigma*), the gradient of the adjoint solve
// (lam), and the chi-update adjoints, the adjoints of sigma^n (written over
// sb1), chi^n (chib_out) and of the velocity gradient L (Lb, 9 per cell,
// row-major).  w_work weighs the step's plastic work 2 D^pl sbar dt h^3.
__global__ void k_adj_predict(StepParams p, StzConst c, const double *__restrict__ v,
                              const double *__restrict__ lam, const double *__restrict__ sig,
                              const double *__restrict__ chi, double *__restrict__ sb1,
                              const double *__restrict__ chib, const double *__restrict__ Db_in,
                              const double *__restrict__ sbb_in, const double *__restrict__ sgb,
                              double *__restrict__ chib_out, double *__restrict__ Lb,
                              double w_work, long nc) {
    CellColumn C;
    if (!cell_column(p.nx, p.ny, p.nz, C)) return;
    const double inv4h = 0.25 / p.h, dt = p.dt, mu = p.mu;
    const double rhs_scale = p.h * p.h / (p.mu * dt);  // (h^2/(mu dt)) / (4h) * 4h
    const double work = w_work * 2.0 * dt * p.h * p.h * p.h;
    GradPlane vlo = grad_plane(v, C.cs, C.k0 * C.pl, C.r0, C.r1, C.i, C.i1);
    GradPlane llo = grad_plane(lam, C.cs, C.k0 * C.pl, C.r0, C.r1, C.i, C.i1);
    for (int k = C.k0; k < C.k1; k++) {
        const GradPlane vhi = grad_plane(v, C.cs, (k + 1) * C.pl, C.r0, C.r1, C.i, C.i1);
        const GradPlane lhi = grad_plane(lam, C.cs, (k + 1) * C.pl, C.r0, C.r1, C.i, C.i1);
        const long q = k * C.pl + C.r0 + C.i;
        double L[3][3], Gl[3][3];
        grad_cell(vlo, vhi, inv4h, L);
        grad_cell(llo, lhi, inv4h, Gl);
        vlo = vhi;
        llo = lhi;
        double s6[6], ss[6];
#pragma unroll
        for (int n = 0; n < 6; n++) {
            s6[n] = sig[n * nc + q];
            ss[n] = sb1[n * nc + q];
        }
        // right-hand side b = (h^2/(mu dt)) corner-div sigma*: its transpose
        // is -(h^2/(mu dt)) times the cell gradient of the solve's adjoint
        ss[0] -= rhs_scale * Gl[0][0];
        ss[1] -= rhs_scale * Gl[1][1];
        ss[2] -= rhs_scale * Gl[2][2];
        ss[3] -= rhs_scale * (Gl[1][2] + Gl[2][1]);
        ss[4] -= rhs_scale * (Gl[0][2] + Gl[2][0]);
        ss[5] -= rhs_scale * (Gl[0][1] + Gl[1][0]);
        // full-matrix adjoint of sigma*
        const double B[3][3] = {{ss[0], 0.5 * ss[5], 0.5 * ss[4]},
                                {0.5 * ss[5], ss[1], 0.5 * ss[3]},
                                {0.5 * ss[4], 0.5 * ss[3], ss[2]}};
        const double S[3][3] = {{s6[0], s6[5], s6[4]}, {s6[5], s6[1], s6[3]}, {s6[4], s6[3], s6[2]}};
        double S0[3][3], sb, inv;
        dev_of(s6, S0, sb, inv);
        double D, Ds, Dc;
        stz_rate_d(c, sb, inv, chi[q], D, Ds, Dc);
        double db = Db_in[q] + work * sb;
        double sbv = sbb_in[q] + work * D;
        const double trL = L[0][0] + L[1][1] + L[2][2];
        const double P = 2.0 * mu * dt * D * inv;
        const double trB = (B[0][0] + B[1][1] + B[2][2]) * (1.0 / 3.0);
        double Sb[3][3], Lbar[3][3];
        double BdotS = 0.0, BdotS0 = 0.0;
#pragma unroll
        for (int a = 0; a < 3; a++)
#pragma unroll
            for (int b = 0; b < 3; b++) {
                BdotS += B[a][b] * S[a][b];
                BdotS0 += B[a][b] * S0[a][b];
            }
#pragma unroll
        for (int a = 0; a < 3; a++)
#pragma unroll
            for (int b = 0; b < 3; b++) {
                double ltb = 0.0, bl = 0.0, bs = 0.0;
#pragma unroll
                for (int e = 0; e < 3; e++) {
                    ltb += L[e][a] * B[e][b];
                    bl += B[a][e] * L[e][b];
                    bs += B[a][e] * S[e][b];
                }
                Sb[a][b] = B[a][b] + dt * (ltb + bl - trL * B[a][b]) -
                           P * (B[a][b] - (a == b ? trB : 0.0));
                Lbar[a][b] = dt * (2.0 * bs - (a == b ? BdotS : 0.0));
            }
        const double Pb = -BdotS0;
        db += Pb * 2.0 * mu * dt * inv;
        sbv -= Pb * 2.0 * mu * dt * D * inv * inv;
        sbv += db * Ds;
        chib_out[q] = chib[q] + db * Dc;
        double out[6];
#pragma unroll
        for (int n = 0; n < 6; n++) out[n] = sgb[n * nc + q];
        const double w = sbv * 0.5 * inv;
#pragma unroll
        for (int a = 0; a < 3; a++)
#pragma unroll
            for (int b = 0; b < 3; b++) Sb[a][b] += w * S0[a][b];
        add_stored(out, Sb, 1.0);
#pragma unroll
        for (int n = 0; n < 6; n++) sb1[n * nc + q] = out[n];
#pragma unroll
        for (int a = 0; a < 3; a++)
#pragma unroll
            for (int b = 0; b < 3; b++) Lb[(a * 3 + b) * nc + q] = Lbar[a][b];
    }
}

// cell tensors read as full 3 x 3 matrices: the stored adjoint of
// sigma^{n+1} mapped through C (C:Sigmabar, symmetric), or a general one
// stored row-major in 9 arrays
struct LoadCSym {
    const double *sb;
    long nc;
    double lam, mu;
    __device__ __forceinline__ void operator()(long q, double T[3][3]) const {
        const double s0 = sb[q], s1 = sb[nc + q], s2 = sb[2 * nc + q];
        const double tr = s0 + s1 + s2;
        T[0][0] = lam * tr + 2.0 * mu * s0;
        T[1][1] = lam * tr + 2.0 * mu * s1;
        T[2][2] = lam * tr + 2.0 * mu * s2;
        T[1][2] = T[2][1] = mu * sb[3 * nc + q];
        T[0][2] = T[2][0] = mu * sb[4 * nc + q];
        T[0][1] = T[1][0] = mu * sb[5 * nc + q];
    }
};
struct LoadFull {
    const double *t;
    long nc;
    __device__ __forceinline__ void operator()(long q, double T[3][3]) const {
#pragma unroll
        for (int a = 0; a < 3; a++)
#pragma unroll
            for (int b = 0; b < 3; b++) T[a][b] = t[(a * 3 + b) * nc + q];
    }
};

// the corner divergence of k_div_rhs for a general cell tensor T (row a =
// output component): the 4 cells (jm..j, im..i) of one cell layer
template <class Load>
__device__ __forceinline__ DivLayer tensor_layer(const Load &ld, long base, long rj0, long rj1,
                                                 int im, int i) {
    double T00[3][3], T01[3][3], T10[3][3], T11[3][3];
    ld(base + rj0 + im, T00);
    ld(base + rj0 + i, T01);
    ld(base + rj1 + im, T10);
    ld(base + rj1 + i, T11);
    DivLayer L;
#pragma unroll
    for (int a = 0; a < 3; a++) {
        L.X[a] = (T01[a][0] - T00[a][0]) + (T11[a][0] - T10[a][0]);
        L.Y[a] = (T10[a][1] - T00[a][1]) + (T11[a][1] - T01[a][1]);
        L.Z[a] = (T00[a][2] + T01[a][2]) + (T10[a][2] + T11[a][2]);
    }
    return L;
}

// out = add + scale * corner-div T at the interior corners (wall planes of
// out are left alone); the transpose of the cell gradient of Eq. (31) is
// -1/(4h) times this divergence
template <class Load>
__global__ void k_corner_div(StepParams p, Load ld, const double *__restrict__ add,
                             double *__restrict__ out, double scale) {
    const int nx = p.nx, ny = p.ny, nz = p.nz;
    const int i = blockIdx.x * BX + threadIdx.x, j = blockIdx.y * BY + threadIdx.y;
    if (i >= nx || j >= ny) return;
    const int k0 = 1 + blockIdx.z * kDivChunk;
    const int k1 = k0 + kDivChunk < nz ? k0 + kDivChunk : nz;
    const int im = i ? i - 1 : nx - 1, jm = j ? j - 1 : ny - 1;
    const long pl = (long)nx * ny, cs = (long)(nz + 1) * pl;
    const long rj0 = (long)jm * nx, rj1 = (long)j * nx;
    DivLayer lo = tensor_layer(ld, (long)(k0 - 1) * pl, rj0, rj1, im, i);
    for (int k = k0; k < k1; k++) {
        const DivLayer hi = tensor_layer(ld, (long)k * pl, rj0, rj1, im, i);
        const long node = (long)k * pl + (long)j * nx + i;
#pragma unroll
        for (int a = 0; a < 3; a++) {
            const double d = (lo.X[a] + hi.X[a]) + (lo.Y[a] + hi.Y[a]) + (hi.Z[a] - lo.Z[a]);
            out[a * cs + node] = (add ? add[a * cs + node] : 0.0) + scale * d;
        }
        lo = hi;
    }
}

// sum over cells of a * b into partials[kRedBlocks] (fixed geometry, so the
// total is bitwise reproducible)
__global__ void __launch_bounds__(kRedThreads)
    k_dot_cells(const double *__restrict__ a, const double *__restrict__ b, long n,
                double *__restrict__ partials) {
    __shared__ double red[kRedThreads / 32];
    double acc = 0.0;
    for (long t = (long)blockIdx.x * kRedThreads + threadIdx.x; t < n;
         t += (long)gridDim.x * kRedThreads)
        acc += a[t] * b[t];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int w = 0; w < kRedThreads / 32; w++) s += red[w];
        partials[blockIdx.x] = s;
    }
}

cudaError_t zero_walls(const StepParams &p, double *x, cudaStream_t s) {
    const long pl = (long)p.nx * p.ny, cs = (long)(p.nz + 1) * pl;
    for (int a = 0; a < 3; a++) {
        cudaError_t e = cudaMemsetAsync(x + a * cs, 0, pl * sizeof(double), s);
        if (e != cudaSuccess) return e;
        e = cudaMemsetAsync(x + a * cs + (long)p.nz * pl, 0, pl * sizeof(double), s);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

}  // namespace

cudaError_t adj_correct(const StepParams &p, const double *sb1, const double *vb1,
                        double *rhs_out, cudaStream_t s) {
    const long nc = (long)p.nx * p.ny * p.nz;
    cudaError_t e = zero_walls(p, rhs_out, s);
    if (e != cudaSuccess) return e;
    const LoadCSym ld{sb1, nc, p.lam, p.mu};
    k_corner_div<LoadCSym><<<cell_grid(p.nx, p.ny, (p.nz - 1 + kDivChunk - 1) / kDivChunk),
                             kBlock, 0, s>>>(p, ld, vb1, rhs_out, -p.dt * 0.25 / p.h);
    count_launch();
    return cudaGetLastError();
}

cudaError_t adj_chi(const StepParams &p, const double *sig, const double *chi, const double *dpl,
                    const double *sbar, const double *cb1, double *chib, double *Db, double *sbb,
                    double *sgb, cudaStream_t s) {
    const long nc = (long)p.nx * p.ny * p.nz;
    k_adj_chi<<<cell_grid(p.nx, p.ny, p.nz), kBlock, 0, s>>>(p, stz_const(p), sig, chi, dpl, sbar,
                                                              cb1, chib, Db, sbb, sgb, nc);
    count_launch();
    return cudaGetLastError();
}

cudaError_t adj_predict(const StepParams &p, const double *v, const double *lam,
                        const double *sig, const double *chi, double *sb1, const double *chib,
                        const double *Db, const double *sbb, const double *sgb, double *chib_out,
                        double *Lb, double w_work, cudaStream_t s) {
    const long nc = (long)p.nx * p.ny * p.nz;
    k_adj_predict<<<cell_grid(p.nx, p.ny, (p.nz + kCellChunk - 1) / kCellChunk), kBlock, 0, s>>>(
        p, stz_const(p), v, lam, sig, chi, sb1, chib, Db, sbb, sgb, chib_out, Lb, w_work, nc);
    count_launch();
    return cudaGetLastError();
}

cudaError_t adj_grad_transpose(const StepParams &p, const double *Lb, double *vb,
                               cudaStream_t s) {
    const long nc = (long)p.nx * p.ny * p.nz;
    cudaError_t e = zero_walls(p, vb, s);
    if (e != cudaSuccess) return e;
    const LoadFull ld{Lb, nc};
    k_corner_div<LoadFull><<<cell_grid(p.nx, p.ny, (p.nz - 1 + kDivChunk - 1) / kDivChunk),
                             kBlock, 0, s>>>(p, ld, nullptr, vb, -0.25 / p.h);
    count_launch();
    return cudaGetLastError();
}

cudaError_t dot_cells(const double *a, const double *b, long n, double *partials,
                      cudaStream_t s) {
    k_dot_cells<<<kRedBlocks, kRedThreads, 0, s>>>(a, b, n, partials);
    count_launch();
    return cudaGetLastError();
}

}  // namespace qsmg

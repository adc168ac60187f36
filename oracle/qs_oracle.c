/*
 * qs_oracle.c -- plain FP64 CPU oracle of the quasi-static projection step.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may call this file:
 * only tests/, __graft_entry__.smoke() and bench.py's cpu_baseline /
 * reference arm load it.  It shares no source with the CUDA library.
 *
 * It follows Boffi & Rycroft, "Parallel three-dimensional simulations of
 * quasi-static elastoplastic solids" (arXiv 1904.03808), step by step, in
 * plain loops:
 *   - staggered grid of section 3.4: velocity at cell corners (i, j, k),
 *     k = 0..nz with walls at k = 0 and k = nz; stress and chi at cell
 *     centres; x and y periodic (section 4, Fig. 5);
 *   - staggered centred difference, Eq. (31), and its corner version;
 *   - collocated 3-point second derivative, Eq. (32), and the 4-point mixed
 *     derivative of section 3.4 for the projection operator of Eq. (30);
 *   - athermal STZ rate, Eqs. (20)-(22); effective temperature, Eq. (26);
 *     intermediate stress, Eq. (27); stress correction, Eq. (29);
 *   - geometric multigrid of section 3.6: halving coarsening, linear
 *     interpolation T, restriction R = T^T, Galerkin A_k = R A_{k-1} T
 *     (Eq. 36), V-cycle with 2 pre- and 2 post-smoothing Gauss-Seidel sweeps.
 *
 * Readings where the paper is silent (each also listed in the design notes):
 *   - the operator is the collocated stencil (section 3.4's stencils "to solve
 *     Eq. (30)"), scaled by -h^2/(mu dt) so that it is SPD and dimensionless;
 *   - Gauss-Seidel is 8-colour, colour c = (i&1) + 2(j&1) + 4(k&1); pre-
 *     smoothing visits colours 0..7, post-smoothing 7..0;
 *   - the coarsest grid is solved by a dense Cholesky factorisation;
 *   - the stopping test is ||b - A v||_2 <= tol * ||b_lifted||_2, where
 *     b_lifted is b minus the wall columns applied to the wall values;
 *   - D^pl = 0 for sbar <= s_Y (and for chi <= 0);
 *   - chi diffusion is a conservative 7-point stencil with face-averaged
 *     D^pl; z ghost cells take linearly extrapolated sigma and chi (section 4)
 *     and D^pl evaluated from them;
 *   - the sign of tr(L) sigma is minus (Eqs. 1, 15, 27; also in the explicit
 *     Eq. 25, whose plus is read as a typo);
 *   - explicit method (section 3.2): the momentum balance Eq. (24) is read
 *     as rho (v' - v)/dt = -rho (v.grad) v + div sigma + rho kappa lap v,
 *     kappa a diffusivity (m^2/s; section 4 sets kappa = kappa' h and the
 *     stability limit dt <= h^2 / (6 kappa)); sigma is advected with the mean
 *     of its cell's corner velocities; ghost values two planes beyond a wall
 *     reflect v through the wall value and extrapolate cell fields linearly;
 *   - optional stress advection in the quasi-static predictor (the general
 *     law of section 2 has -(v.grad) sigma; Eq. 27 drops it): the same ENO
 *     advection with the mean corner velocity of v^n and the same ghosts as
 *     the explicit method, added to the rate of Eq. (27).
 *
 * Stencil tables: S[d][a][b] with d = (dz+1)*9 + (dy+1)*3 + (dx+1) for
 * offsets in {-1,0,1}^3, a = output component, b = input component.
 * (A x)_a(p) = sum_d sum_b S[d][a][b] x_b(p + d).
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* ------------------------------------------------------------------ */
/* indexing                                                            */
/* ------------------------------------------------------------------ */

/* corner node (component c, plane k in 0..nz, row j, column i) */
static inline long node(int nx, int ny, int nz, int c, int k, int j, int i)
{
    return (((long)c * (nz + 1) + k) * ny + j) * nx + i;
}

/* cell scalar (k in 0..nz-1) */
static inline long cell(int nx, int ny, int k, int j, int i)
{
    return ((long)k * ny + j) * nx + i;
}

static inline int wrap(int i, int n) { return ((i % n) + n) % n; }

int ora_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* ------------------------------------------------------------------ */
/* projection operator, Eq. (30) with the stencils of section 3.4       */
/* ------------------------------------------------------------------ */

/*
 * (A v)_a = dt [ (lam+2mu) d_aa v_a + mu sum_{b!=a} d_bb v_a
 *              + (lam+mu) sum_{b!=a} d_ab v_b ]
 * with d_aa the 3-point second difference (Eq. 32) and d_ab the 4-point mixed
 * difference.  The oracle stores Ahat = -(h^2/(mu dt)) A, so every entry is a
 * pure number depending on lam/mu only.
 */
void ora_fine_stencil(double lam, double mu, double *S)
{
    double lp = (lam + 2.0 * mu) / mu; /* (lam+2mu)/mu */
    double kp = (lam + mu) / mu;       /* (lam+mu)/mu  */
    memset(S, 0, 243 * sizeof(double));
    for (int a = 0; a < 3; a++) {
        /* centre: -( (lam+2mu)(-2) + mu(-2)(-2 ... ) ) / mu */
        double diag = 0.0;
        for (int ax = 0; ax < 3; ax++)
            diag += 2.0 * (ax == a ? lp : 1.0);
        S[(13 * 3 + a) * 3 + a] = diag;
    }
    /* face neighbours: d_cc couples v_a with itself */
    for (int ax = 0; ax < 3; ax++)
        for (int s = -1; s <= 1; s += 2) {
            int off[3] = {0, 0, 0};
            off[ax] = s;
            int d = (off[2] + 1) * 9 + (off[1] + 1) * 3 + (off[0] + 1);
            for (int a = 0; a < 3; a++)
                S[(d * 3 + a) * 3 + a] = -(ax == a ? lp : 1.0);
        }
    /* edge neighbours: d_ab f = (f++ - f+- - f-+ + f--)/4 couples v_a, v_b */
    for (int a = 0; a < 3; a++)
        for (int b = a + 1; b < 3; b++)
            for (int sa = -1; sa <= 1; sa += 2)
                for (int sb = -1; sb <= 1; sb += 2) {
                    int off[3] = {0, 0, 0};
                    off[a] = sa;
                    off[b] = sb;
                    int d = (off[2] + 1) * 9 + (off[1] + 1) * 3 + (off[0] + 1);
                    double w = -kp * sa * sb / 4.0;
                    S[(d * 3 + a) * 3 + b] = w;
                    S[(d * 3 + b) * 3 + a] = w;
                }
}

/*
 * Galerkin product A_c = R A T (Eq. 36) for a constant stencil on the
 * unbounded lattice:  A_c[I, J] = sum_{p,q} T[p,I] A[p,q] T[q,J]
 * with p = 2I + e, q = 2J + f and the trilinear weights
 * t(e) = prod_axis (e_axis == 0 ? 1 : 1/2).  Hence for D = J - I,
 * A_c(D) = sum_{e,f} t(e) t(f) A(2D + f - e).
 */
static double tw(int e0, int e1, int e2)
{
    return (e0 ? 0.5 : 1.0) * (e1 ? 0.5 : 1.0) * (e2 ? 0.5 : 1.0);
}

void ora_galerkin(const double *Sf, double *Sc)
{
    memset(Sc, 0, 243 * sizeof(double));
    for (int Dz = -1; Dz <= 1; Dz++)
    for (int Dy = -1; Dy <= 1; Dy++)
    for (int Dx = -1; Dx <= 1; Dx++) {
        int dc = (Dz + 1) * 9 + (Dy + 1) * 3 + (Dx + 1);
        for (int ez = -1; ez <= 1; ez++)
        for (int ey = -1; ey <= 1; ey++)
        for (int ex = -1; ex <= 1; ex++)
        for (int fz = -1; fz <= 1; fz++)
        for (int fy = -1; fy <= 1; fy++)
        for (int fx = -1; fx <= 1; fx++) {
            int gx = 2 * Dx + fx - ex, gy = 2 * Dy + fy - ey, gz = 2 * Dz + fz - ez;
            if (gx < -1 || gx > 1 || gy < -1 || gy > 1 || gz < -1 || gz > 1)
                continue;
            int df = (gz + 1) * 9 + (gy + 1) * 3 + (gx + 1);
            double w = tw(ex, ey, ez) * tw(fx, fy, fz);
            for (int a = 0; a < 9; a++)
                Sc[dc * 9 + a] += w * Sf[df * 9 + a];
        }
    }
}

/* y = A x on interior nodes (k = 1..nz-1), using x on the wall planes; the
 * wall planes of y are set to zero. */
void ora_apply(int nx, int ny, int nz, const double *S, const double *x, double *y)
{
#pragma omp parallel for schedule(static)
    for (int k = 1; k < nz; k++)
        for (int j = 0; j < ny; j++)
            for (int i = 0; i < nx; i++) {
                double acc[3] = {0.0, 0.0, 0.0};
                for (int dz = -1; dz <= 1; dz++)
                for (int dy = -1; dy <= 1; dy++)
                for (int dx = -1; dx <= 1; dx++) {
                    int d = (dz + 1) * 9 + (dy + 1) * 3 + (dx + 1);
                    int kk = k + dz, jj = wrap(j + dy, ny), ii = wrap(i + dx, nx);
                    for (int a = 0; a < 3; a++)
                        for (int b = 0; b < 3; b++)
                            acc[a] += S[(d * 3 + a) * 3 + b] * x[node(nx, ny, nz, b, kk, jj, ii)];
                }
                for (int a = 0; a < 3; a++)
                    y[node(nx, ny, nz, a, k, j, i)] = acc[a];
            }
    for (int a = 0; a < 3; a++)
        for (int j = 0; j < ny; j++)
            for (int i = 0; i < nx; i++) {
                y[node(nx, ny, nz, a, 0, j, i)] = 0.0;
                y[node(nx, ny, nz, a, nz, j, i)] = 0.0;
            }
}

/* r = b - A x on interior nodes; zero on the walls */
void ora_residual(int nx, int ny, int nz, const double *S, const double *b,
                  const double *x, double *r)
{
    ora_apply(nx, ny, nz, S, x, r);
    long n = 3L * (nz + 1) * ny * nx;
    for (long p = 0; p < n; p++)
        r[p] = -r[p];
    for (int a = 0; a < 3; a++)
        for (int k = 1; k < nz; k++)
            for (int j = 0; j < ny; j++)
                for (int i = 0; i < nx; i++) {
                    long p = node(nx, ny, nz, a, k, j, i);
                    r[p] += b[p];
                }
}

/* sum of squares over interior nodes, serial so the order is fixed */
double ora_norm2(int nx, int ny, int nz, const double *r)
{
    double s = 0.0;
    for (int a = 0; a < 3; a++)
        for (int k = 1; k < nz; k++)
            for (int j = 0; j < ny; j++)
                for (int i = 0; i < nx; i++) {
                    double v = r[node(nx, ny, nz, a, k, j, i)];
                    s += v * v;
                }
    return s;
}

/* solve the symmetric 3x3 system M y = f by Gaussian elimination */
static void solve3(const double *M, const double *f, double *y)
{
    double A[3][4];
    for (int a = 0; a < 3; a++) {
        for (int b = 0; b < 3; b++)
            A[a][b] = M[a * 3 + b];
        A[a][3] = f[a];
    }
    for (int p = 0; p < 3; p++)
        for (int q = p + 1; q < 3; q++) {
            double m = A[q][p] / A[p][p];
            for (int c = p; c < 4; c++)
                A[q][c] -= m * A[p][c];
        }
    for (int p = 2; p >= 0; p--) {
        double s = A[p][3];
        for (int c = p + 1; c < 3; c++)
            s -= A[p][c] * y[c];
        y[p] = s / A[p][p];
    }
}

/* one Gauss-Seidel pass over the nodes of one colour (block GS, 3x3 blocks):
 * x_p <- A_pp^{-1} (b_p - sum_{q != p} A_pq x_q) with current neighbours. */
void ora_gs_colour(int nx, int ny, int nz, const double *S, const double *b,
                   double *x, int colour)
{
    int pi = colour & 1, pj = (colour >> 1) & 1, pk = (colour >> 2) & 1;
    int k0 = (pk == 1) ? 1 : 2;
#pragma omp parallel for schedule(static)
    for (int k = k0; k < nz; k += 2)
        for (int j = pj; j < ny; j += 2)
            for (int i = pi; i < nx; i += 2) {
                double f[3];
                for (int a = 0; a < 3; a++)
                    f[a] = b[node(nx, ny, nz, a, k, j, i)];
                for (int dz = -1; dz <= 1; dz++)
                for (int dy = -1; dy <= 1; dy++)
                for (int dx = -1; dx <= 1; dx++) {
                    int d = (dz + 1) * 9 + (dy + 1) * 3 + (dx + 1);
                    if (d == 13)
                        continue;
                    int kk = k + dz, jj = wrap(j + dy, ny), ii = wrap(i + dx, nx);
                    for (int a = 0; a < 3; a++)
                        for (int c = 0; c < 3; c++)
                            f[a] -= S[(d * 3 + a) * 3 + c] * x[node(nx, ny, nz, c, kk, jj, ii)];
                }
                double y[3];
                solve3(S + 13 * 9, f, y);
                for (int a = 0; a < 3; a++)
                    x[node(nx, ny, nz, a, k, j, i)] = y[a];
            }
}

/* restriction R = T^T: bc(I) = sum_e t(e) r(2I + e), coarse interior only */
void ora_restrict(int nx, int ny, int nz, const double *r, double *bc)
{
    int cx = nx / 2, cy = ny / 2, cz = nz / 2;
    memset(bc, 0, 3L * (cz + 1) * cy * cx * sizeof(double));
#pragma omp parallel for schedule(static)
    for (int K = 1; K < cz; K++)
        for (int J = 0; J < cy; J++)
            for (int I = 0; I < cx; I++)
                for (int a = 0; a < 3; a++) {
                    double s = 0.0;
                    for (int ez = -1; ez <= 1; ez++)
                    for (int ey = -1; ey <= 1; ey++)
                    for (int ex = -1; ex <= 1; ex++)
                        s += tw(ex, ey, ez) *
                             r[node(nx, ny, nz, a, 2 * K + ez, wrap(2 * J + ey, ny), wrap(2 * I + ex, nx))];
                    bc[node(cx, cy, cz, a, K, J, I)] = s;
                }
}

/* prolongation x += T xc: linear interpolation, coarse node I sits at fine 2I;
 * coarse wall planes carry zero correction. */
void ora_prolong_add(int nx, int ny, int nz, const double *xc, double *x)
{
    int cx = nx / 2, cy = ny / 2, cz = nz / 2;
#pragma omp parallel for schedule(static)
    for (int k = 1; k < nz; k++)
        for (int j = 0; j < ny; j++)
            for (int i = 0; i < nx; i++) {
                /* contributing coarse indices and weights along each axis */
                int Ks[2], Js[2], Is[2], nk, nj, ni;
                double wk[2], wj[2], wi[2];
                if (k % 2 == 0) { Ks[0] = k / 2; wk[0] = 1.0; nk = 1; }
                else { Ks[0] = (k - 1) / 2; Ks[1] = (k + 1) / 2; wk[0] = wk[1] = 0.5; nk = 2; }
                if (j % 2 == 0) { Js[0] = j / 2; wj[0] = 1.0; nj = 1; }
                else { Js[0] = (j - 1) / 2; Js[1] = wrap((j + 1) / 2, cy); wj[0] = wj[1] = 0.5; nj = 2; }
                if (i % 2 == 0) { Is[0] = i / 2; wi[0] = 1.0; ni = 1; }
                else { Is[0] = (i - 1) / 2; Is[1] = wrap((i + 1) / 2, cx); wi[0] = wi[1] = 0.5; ni = 2; }
                for (int a = 0; a < 3; a++) {
                    double s = 0.0;
                    for (int p = 0; p < nk; p++) {
                        if (Ks[p] == 0 || Ks[p] == cz)
                            continue; /* homogeneous Dirichlet correction */
                        for (int q = 0; q < nj; q++)
                            for (int t = 0; t < ni; t++)
                                s += wk[p] * wj[q] * wi[t] * xc[node(cx, cy, cz, a, Ks[p], Js[q], Is[t])];
                    }
                    x[node(nx, ny, nz, a, k, j, i)] += s;
                }
            }
}

/* ------------------------------------------------------------------ */
/* multigrid hierarchy (section 3.6)                                   */
/* ------------------------------------------------------------------ */

#define ORA_MAXLEV 16

typedef struct ora_mg {
    int nlev;
    int dims[ORA_MAXLEV][3];
    double S[ORA_MAXLEV][243];
    double *x[ORA_MAXLEV], *b[ORA_MAXLEV], *r[ORA_MAXLEV];
    int nu1, nu2;
    int ncoarse;     /* unknowns on the coarsest level */
    double *chol;    /* lower Cholesky factor, row-major ncoarse^2 */
    double *cwork;
} ora_mg;

/* coarsen while every dimension is even and its half is still >= 4 */
static int can_coarsen(const int *d)
{
    for (int a = 0; a < 3; a++)
        if (d[a] % 2 != 0 || d[a] / 2 < 4)
            return 0;
    return 1;
}

/* interior unknown number of (component a, plane k, row j, column i) */
static long unk(int nx, int ny, int a, int k, int j, int i)
{
    return (((long)(k - 1) * ny + j) * nx + i) * 3 + a;
}

int ora_mg_coarse_size(ora_mg *m) { return m->ncoarse; }

/* dense matrix of the coarsest operator (interior unknowns only) */
static void assemble_dense(int nx, int ny, int nz, const double *S, double *Ad)
{
    long n = 3L * nx * ny * (nz - 1);
    memset(Ad, 0, n * n * sizeof(double));
    for (int k = 1; k < nz; k++)
        for (int j = 0; j < ny; j++)
            for (int i = 0; i < nx; i++)
                for (int dz = -1; dz <= 1; dz++)
                for (int dy = -1; dy <= 1; dy++)
                for (int dx = -1; dx <= 1; dx++) {
                    int kk = k + dz;
                    if (kk < 1 || kk > nz - 1)
                        continue; /* wall columns are not unknowns */
                    int d = (dz + 1) * 9 + (dy + 1) * 3 + (dx + 1);
                    int jj = wrap(j + dy, ny), ii = wrap(i + dx, nx);
                    for (int a = 0; a < 3; a++)
                        for (int c = 0; c < 3; c++)
                            Ad[unk(nx, ny, a, k, j, i) * n + unk(nx, ny, c, kk, jj, ii)] +=
                                S[(d * 3 + a) * 3 + c];
                }
}

/* dense matrix of level l (tests use it for small direct solves) */
int ora_mg_dense(ora_mg *m, int l, double *Ad)
{
    int *d = m->dims[l];
    assemble_dense(d[0], d[1], d[2], m->S[l], Ad);
    return 3 * d[0] * d[1] * (d[2] - 1);
}

/* in-place lower Cholesky factor; returns 0 on success, -1 if not SPD */
static int cholesky(double *A, long n)
{
    for (long j = 0; j < n; j++) {
        double s = A[j * n + j];
        for (long p = 0; p < j; p++)
            s -= A[j * n + p] * A[j * n + p];
        if (!(s > 0.0))
            return -1;
        double ljj = sqrt(s);
        A[j * n + j] = ljj;
        for (long i = j + 1; i < n; i++) {
            double t = A[i * n + j];
            for (long p = 0; p < j; p++)
                t -= A[i * n + p] * A[j * n + p];
            A[i * n + j] = t / ljj;
        }
        for (long i = 0; i < j; i++)
            A[i * n + j] = 0.0;
    }
    return 0;
}

/* free helper usable from Python: Cholesky of a dense SPD matrix */
int ora_cholesky(double *A, long n) { return cholesky(A, n); }

static void chol_solve(const double *L, long n, double *y)
{
    for (long i = 0; i < n; i++) {
        double s = y[i];
        for (long p = 0; p < i; p++)
            s -= L[i * n + p] * y[p];
        y[i] = s / L[i * n + i];
    }
    for (long i = n - 1; i >= 0; i--) {
        double s = y[i];
        for (long p = i + 1; p < n; p++)
            s -= L[p * n + i] * y[p];
        y[i] = s / L[i * n + i];
    }
}

void ora_mg_free(ora_mg *m)
{
    if (!m)
        return;
    for (int l = 0; l < m->nlev; l++) {
        free(m->x[l]);
        free(m->b[l]);
        free(m->r[l]);
    }
    free(m->chol);
    free(m->cwork);
    free(m);
}

/* returns NULL for unsupported shapes: nx, ny even >= 4, nz even >= 2, and
 * at most 3072 unknowns on the coarsest level */
ora_mg *ora_mg_create(int nx, int ny, int nz, double lam, double mu, int nu1, int nu2)
{
    if (nx < 4 || ny < 4 || nz < 2 || nx % 2 || ny % 2 || nz % 2)
        return NULL;
    ora_mg *m = (ora_mg *)calloc(1, sizeof(ora_mg));
    m->nu1 = nu1;
    m->nu2 = nu2;
    m->dims[0][0] = nx;
    m->dims[0][1] = ny;
    m->dims[0][2] = nz;
    m->nlev = 1;
    while (m->nlev < ORA_MAXLEV && can_coarsen(m->dims[m->nlev - 1])) {
        for (int a = 0; a < 3; a++)
            m->dims[m->nlev][a] = m->dims[m->nlev - 1][a] / 2;
        m->nlev++;
    }
    ora_fine_stencil(lam, mu, m->S[0]);
    for (int l = 1; l < m->nlev; l++)
        ora_galerkin(m->S[l - 1], m->S[l]);
    for (int l = 0; l < m->nlev; l++) {
        int *d = m->dims[l];
        long n = 3L * (d[2] + 1) * d[1] * d[0];
        m->x[l] = (double *)calloc(n, sizeof(double));
        m->b[l] = (double *)calloc(n, sizeof(double));
        m->r[l] = (double *)calloc(n, sizeof(double));
    }
    int *dc = m->dims[m->nlev - 1];
    long nc = 3L * dc[0] * dc[1] * (dc[2] - 1);
    if (nc > 3072) {
        ora_mg_free(m);
        return NULL;
    }
    m->ncoarse = (int)nc;
    m->chol = (double *)malloc(nc * nc * sizeof(double));
    m->cwork = (double *)malloc(nc * sizeof(double));
    assemble_dense(dc[0], dc[1], dc[2], m->S[m->nlev - 1], m->chol);
    if (cholesky(m->chol, nc) != 0) {
        ora_mg_free(m);
        return NULL;
    }
    return m;
}

int ora_mg_levels(ora_mg *m) { return m->nlev; }

void ora_mg_level_dims(ora_mg *m, int l, int *d)
{
    for (int a = 0; a < 3; a++)
        d[a] = m->dims[l][a];
}

void ora_mg_stencil(ora_mg *m, int l, double *S)
{
    memcpy(S, m->S[l], 243 * sizeof(double));
}

/* coarsest level: x += A^{-1} (b - A x) by the dense Cholesky factor */
static void coarse_solve(ora_mg *m, int l, const double *b, double *x)
{
    int nx = m->dims[l][0], ny = m->dims[l][1], nz = m->dims[l][2];
    ora_residual(nx, ny, nz, m->S[l], b, x, m->r[l]);
    for (int k = 1; k < nz; k++)
        for (int j = 0; j < ny; j++)
            for (int i = 0; i < nx; i++)
                for (int a = 0; a < 3; a++)
                    m->cwork[unk(nx, ny, a, k, j, i)] = m->r[l][node(nx, ny, nz, a, k, j, i)];
    chol_solve(m->chol, m->ncoarse, m->cwork);
    for (int k = 1; k < nz; k++)
        for (int j = 0; j < ny; j++)
            for (int i = 0; i < nx; i++)
                for (int a = 0; a < 3; a++)
                    x[node(nx, ny, nz, a, k, j, i)] += m->cwork[unk(nx, ny, a, k, j, i)];
}

/* one V-cycle on level l for A_l x = b (x, b of level l) */
static void vcycle(ora_mg *m, int l, const double *b, double *x)
{
    int nx = m->dims[l][0], ny = m->dims[l][1], nz = m->dims[l][2];
    if (l == m->nlev - 1) {
        coarse_solve(m, l, b, x);
        return;
    }
    for (int s = 0; s < m->nu1; s++)
        for (int c = 0; c < 8; c++)
            ora_gs_colour(nx, ny, nz, m->S[l], b, x, c);
    ora_residual(nx, ny, nz, m->S[l], b, x, m->r[l]);
    ora_restrict(nx, ny, nz, m->r[l], m->b[l + 1]);
    int *dc = m->dims[l + 1];
    memset(m->x[l + 1], 0, 3L * (dc[2] + 1) * dc[1] * dc[0] * sizeof(double));
    vcycle(m, l + 1, m->b[l + 1], m->x[l + 1]);
    ora_prolong_add(nx, ny, nz, m->x[l + 1], x);
    for (int s = 0; s < m->nu2; s++)
        for (int c = 7; c >= 0; c--)
            ora_gs_colour(nx, ny, nz, m->S[l], b, x, c);
}

void ora_mg_vcycle(ora_mg *m, const double *b, double *x) { vcycle(m, 0, b, x); }

/*
 * Solve A v = b on the fine level: V-cycles until
 * ||b - A v|| <= tol ||b_lifted||, at most max_cycles.  With tol <= 0 exactly
 * max_cycles cycles run.  hist receives the relative residual before the
 * first cycle and after each cycle (max_cycles + 1 entries).
 * Returns 0 ok, 5 not converged, 6 non-finite residual.
 */
int ora_mg_solve(ora_mg *m, const double *b, double *x, double tol, int max_cycles,
                 int *cycles, double *hist)
{
    int nx = m->dims[0][0], ny = m->dims[0][1], nz = m->dims[0][2];
    long n = 3L * (nz + 1) * ny * nx;
    double *r = m->r[0];
    /* lifted right-hand side: b - A (walls of x, zero interior) */
    double *w = (double *)calloc(n, sizeof(double));
    for (int a = 0; a < 3; a++)
        for (int j = 0; j < ny; j++)
            for (int i = 0; i < nx; i++) {
                w[node(nx, ny, nz, a, 0, j, i)] = x[node(nx, ny, nz, a, 0, j, i)];
                w[node(nx, ny, nz, a, nz, j, i)] = x[node(nx, ny, nz, a, nz, j, i)];
            }
    ora_residual(nx, ny, nz, m->S[0], b, w, r);
    free(w);
    double bnorm = sqrt(ora_norm2(nx, ny, nz, r));
    *cycles = 0;
    if (bnorm == 0.0) {
        for (int a = 0; a < 3; a++)
            for (int k = 1; k < nz; k++)
                for (int j = 0; j < ny; j++)
                    for (int i = 0; i < nx; i++)
                        x[node(nx, ny, nz, a, k, j, i)] = 0.0;
        if (hist)
            hist[0] = 0.0;
        return 0;
    }
    ora_residual(nx, ny, nz, m->S[0], b, x, r);
    double rel = sqrt(ora_norm2(nx, ny, nz, r)) / bnorm;
    if (hist)
        hist[0] = rel;
    int it = 0;
    for (;;) {
        if (!isfinite(rel)) {
            *cycles = it;
            return 6;
        }
        if (tol > 0.0 && rel <= tol)
            break;
        if (it >= max_cycles) {
            *cycles = it;
            return tol > 0.0 ? 5 : 0;
        }
        vcycle(m, 0, b, x);
        it++;
        ora_residual(nx, ny, nz, m->S[0], b, x, r);
        rel = sqrt(ora_norm2(nx, ny, nz, r)) / bnorm;
        if (hist)
            hist[it] = rel;
    }
    *cycles = it;
    return 0;
}

/* ------------------------------------------------------------------ */
/* pointwise stress / STZ / chi update (sections 3.1, 3.3)             */
/* ------------------------------------------------------------------ */

typedef struct {
    double tau0, eps0, c0, Delta_K, Omega, T, chi_inf, ez_K, sY, l, kB;
} ora_stz;

typedef struct {
    int kind; /* 0 simple shear, 1 disc top, 2 disc top and bottom, 3 anti-rotating */
    double U_B, t_ramp, omega, R, lambda_w;
} ora_bc;

/* athermal STZ rate magnitude, Eqs. (20)-(22); zero at or below yield */
double ora_dpl(const ora_stz *p, double sbar, double chi)
{
    if (!(sbar > p->sY) || !(chi > 0.0))
        return 0.0;
    double C = exp(-p->Delta_K / p->T) * cosh(p->Omega * p->eps0 * sbar / (p->kB * p->T));
    return exp(-p->ez_K / chi) * C * (1.0 - p->sY / sbar) / p->tau0;
}

/* stress components stored xx,yy,zz,yz,xz,xy; full symmetric matrix */
static void sym_full(const double *s6, double s[3][3])
{
    s[0][0] = s6[0]; s[1][1] = s6[1]; s[2][2] = s6[2];
    s[1][2] = s[2][1] = s6[3];
    s[0][2] = s[2][0] = s6[4];
    s[0][1] = s[1][0] = s6[5];
}

/* sbar with sbar^2 = 1/2 sum_ij sigma0_ij^2 (section 3.1) */
static double sbar_of(const double s[3][3])
{
    double tr3 = (s[0][0] + s[1][1] + s[2][2]) / 3.0;
    double q = 0.0;
    for (int a = 0; a < 3; a++)
        for (int b = 0; b < 3; b++) {
            double d = s[a][b] - (a == b ? tr3 : 0.0);
            q += d * d;
        }
    return sqrt(0.5 * q);
}

/* staggered centred difference, Eq. (31): L[a][b] = d v_a / d x_b at cell
 * centre (i+1/2, j+1/2, k+1/2) from its 8 corners */
static void cell_grad(int nx, int ny, int nz, const double *v, double h, int k, int j, int i,
                      double L[3][3])
{
    int i1 = wrap(i + 1, nx), j1 = wrap(j + 1, ny);
    for (int a = 0; a < 3; a++) {
#define V(kk, jj, ii) v[node(nx, ny, nz, a, kk, jj, ii)]
        double dx = V(k, j, i1) - V(k, j, i) + V(k, j1, i1) - V(k, j1, i) + V(k + 1, j, i1) -
                    V(k + 1, j, i) + V(k + 1, j1, i1) - V(k + 1, j1, i);
        double dy = V(k, j1, i) - V(k, j, i) + V(k, j1, i1) - V(k, j, i1) + V(k + 1, j1, i) -
                    V(k + 1, j, i) + V(k + 1, j1, i1) - V(k + 1, j, i1);
        double dz = V(k + 1, j, i) - V(k, j, i) + V(k + 1, j1, i) - V(k, j1, i) + V(k + 1, j, i1) -
                    V(k, j, i1) + V(k + 1, j1, i1) - V(k, j1, i1);
#undef V
        L[a][0] = dx / (4.0 * h);
        L[a][1] = dy / (4.0 * h);
        L[a][2] = dz / (4.0 * h);
    }
}

/* Eq. (31) at every cell: L (9 per cell, row-major a,b), exposed for tests */
void ora_cell_gradient(int nx, int ny, int nz, double h, const double *v, double *Lout)
{
    for (int k = 0; k < nz; k++)
        for (int j = 0; j < ny; j++)
            for (int i = 0; i < nx; i++) {
                double L[3][3];
                cell_grad(nx, ny, nz, v, h, k, j, i, L);
                for (int a = 0; a < 9; a++)
                    Lout[cell(nx, ny, k, j, i) * 9 + a] = L[a / 3][a % 3];
            }
}


double ora_eno(const double *f, double u, double h);
static double cell_val(const double *f, int nx, int ny, int nz, int kk, int j, int i);

/*
 * Intermediate stress, Eq. (27), with D^pl of the same state:
 *   sigma* = sigma + dt (L sigma + sigma L^T - tr(L) sigma - C:(D^pl sigma0/sbar))
 * with C:X = lam tr(X) I + 2 mu X; sigma0 is traceless, so the plastic term
 * is 2 mu D^pl sigma0 / sbar.  Writes sigma* (6 per cell, same layout as
 * sigma), D^pl and sbar per cell.
 * With advect != 0 the rate also holds the advection -(u.grad) sigma of the
 * general constitutive law (section 2, the form Eq. 27 drops): u the mean of
 * the cell's 8 corner velocities of v^n, the derivatives by ENO (Eq. 33) with
 * the cell ghosts of the explicit method (linear extrapolation beyond the z
 * boundaries; x and y wrap).
 */
void ora_stress_star_adv(int nx, int ny, int nz, double h, double dt, double mu,
                         const ora_stz *p, const double *v, const double *sig, const double *chi,
                         double *sig_star, double *dpl, double *sbar_out, int advect)
{
    static const int comp[3][3] = {{0, 5, 4}, {5, 1, 3}, {4, 3, 2}};
    long nc = (long)nx * ny * nz;
#pragma omp parallel for schedule(static)
    for (int k = 0; k < nz; k++)
        for (int j = 0; j < ny; j++)
            for (int i = 0; i < nx; i++) {
                long q = cell(nx, ny, k, j, i);
                double s6[6], s[3][3], L[3][3], rate[3][3], adv[6] = {0, 0, 0, 0, 0, 0};
                for (int c = 0; c < 6; c++)
                    s6[c] = sig[c * nc + q];
                sym_full(s6, s);
                cell_grad(nx, ny, nz, v, h, k, j, i, L);
                if (advect) {
                    double u[3] = {0.0, 0.0, 0.0};
                    for (int a = 0; a < 3; a++)
                        for (int dk = 0; dk < 2; dk++)
                            for (int dj = 0; dj < 2; dj++)
                                for (int di = 0; di < 2; di++)
                                    u[a] += 0.125 * v[node(nx, ny, nz, a, k + dk, wrap(j + dj, ny),
                                                           wrap(i + di, nx))];
                    for (int c = 0; c < 6; c++) {
                        const double *f = sig + c * nc;
                        double fx[5], fy[5], fz[5];
                        for (int m = -2; m <= 2; m++) {
                            fx[m + 2] = f[cell(nx, ny, k, j, wrap(i + m, nx))];
                            fy[m + 2] = f[cell(nx, ny, k, wrap(j + m, ny), i)];
                            fz[m + 2] = cell_val(f, nx, ny, nz, k + m, j, i);
                        }
                        adv[c] = u[0] * ora_eno(fx, u[0], h) + u[1] * ora_eno(fy, u[1], h) +
                                 u[2] * ora_eno(fz, u[2], h);
                    }
                }
                double sb = sbar_of(s);
                double D = ora_dpl(p, sb, chi[q]);
                double trL = L[0][0] + L[1][1] + L[2][2];
                double tr3 = (s[0][0] + s[1][1] + s[2][2]) / 3.0;
                for (int a = 0; a < 3; a++)
                    for (int b = 0; b < 3; b++) {
                        double r = advect ? -adv[comp[a][b]] - trL * s[a][b] : -trL * s[a][b];
                        for (int c = 0; c < 3; c++)
                            r += L[a][c] * s[c][b] + s[a][c] * L[b][c];
                        if (D > 0.0)
                            r -= 2.0 * mu * D * (s[a][b] - (a == b ? tr3 : 0.0)) / sb;
                        rate[a][b] = r;
                    }
                sig_star[0 * nc + q] = s[0][0] + dt * rate[0][0];
                sig_star[1 * nc + q] = s[1][1] + dt * rate[1][1];
                sig_star[2 * nc + q] = s[2][2] + dt * rate[2][2];
                sig_star[3 * nc + q] = s[1][2] + dt * rate[1][2];
                sig_star[4 * nc + q] = s[0][2] + dt * rate[0][2];
                sig_star[5 * nc + q] = s[0][1] + dt * rate[0][1];
                dpl[q] = D;
                sbar_out[q] = sb;
            }
}

void ora_stress_star(int nx, int ny, int nz, double h, double dt, double mu,
                     const ora_stz *p, const double *v, const double *sig, const double *chi,
                     double *sig_star, double *dpl, double *sbar_out)
{
    ora_stress_star_adv(nx, ny, nz, h, dt, mu, p, v, sig, chi, sig_star, dpl, sbar_out, 0);
}

/* D^pl of a z ghost cell: sigma and chi linearly extrapolated from the two
 * nearest layers (section 4: fields stay free at the z boundaries) */
static double ghost_dpl(int nx, int ny, const ora_stz *p, const double *sig, const double *chi,
                        long nc, int k0, int k1, int j, int i, double *chi_g)
{
    double s6[6], s[3][3];
    long q0 = cell(nx, ny, k0, j, i), q1 = cell(nx, ny, k1, j, i);
    for (int c = 0; c < 6; c++)
        s6[c] = 2.0 * sig[c * nc + q0] - sig[c * nc + q1];
    sym_full(s6, s);
    *chi_g = 2.0 * chi[q0] - chi[q1];
    return ora_dpl(p, sbar_of(s), *chi_g);
}

/*
 * Effective temperature, Eq. (26) (forward Euler of Eq. 23):
 *   chi' = chi + (dt/c0) [ (D^pl:sigma0 / s_Y)(chi_inf - chi) + l^2 div(D^pl grad chi) ]
 * with D^pl:sigma0 = 2 D^pl sbar and the diffusion as a conservative 7-point
 * sum with face coefficients (D_P + D_N)/2.  sig, chi, dpl, sbar are the
 * state at step n.
 */
void ora_chi_update(int nx, int ny, int nz, double h, double dt, const ora_stz *p,
                    const double *sig, const double *chi, const double *dpl,
                    const double *sbar, double *chi_new)
{
    long nc = (long)nx * ny * nz;
    double lh2 = (p->l * p->l) / (h * h);
#pragma omp parallel for schedule(static)
    for (int k = 0; k < nz; k++)
        for (int j = 0; j < ny; j++)
            for (int i = 0; i < nx; i++) {
                long q = cell(nx, ny, k, j, i);
                double c0 = chi[q], D0 = dpl[q];
                double nb_chi[6], nb_D[6];
                int ip = wrap(i + 1, nx), im = wrap(i - 1, nx);
                int jp = wrap(j + 1, ny), jm = wrap(j - 1, ny);
                nb_chi[0] = chi[cell(nx, ny, k, j, ip)]; nb_D[0] = dpl[cell(nx, ny, k, j, ip)];
                nb_chi[1] = chi[cell(nx, ny, k, j, im)]; nb_D[1] = dpl[cell(nx, ny, k, j, im)];
                nb_chi[2] = chi[cell(nx, ny, k, jp, i)]; nb_D[2] = dpl[cell(nx, ny, k, jp, i)];
                nb_chi[3] = chi[cell(nx, ny, k, jm, i)]; nb_D[3] = dpl[cell(nx, ny, k, jm, i)];
                if (k + 1 < nz) {
                    nb_chi[4] = chi[cell(nx, ny, k + 1, j, i)];
                    nb_D[4] = dpl[cell(nx, ny, k + 1, j, i)];
                } else {
                    nb_D[4] = ghost_dpl(nx, ny, p, sig, chi, nc, nz - 1, nz - 2, j, i, &nb_chi[4]);
                }
                if (k > 0) {
                    nb_chi[5] = chi[cell(nx, ny, k - 1, j, i)];
                    nb_D[5] = dpl[cell(nx, ny, k - 1, j, i)];
                } else {
                    nb_D[5] = ghost_dpl(nx, ny, p, sig, chi, nc, 0, 1, j, i, &nb_chi[5]);
                }
                double diff = 0.0;
                for (int n = 0; n < 6; n++)
                    diff += 0.5 * (D0 + nb_D[n]) * (nb_chi[n] - c0);
                double growth = 2.0 * D0 * sbar[q] / p->sY * (p->chi_inf - c0);
                chi_new[q] = c0 + dt / p->c0 * (growth + lh2 * diff);
            }
}

/*
 * Right-hand side of the scaled projection system: b = (h^2/(mu dt)) div sigma*
 * at interior corners (Eq. 30 with the operator scaled by -h^2/(mu dt)).  The
 * corner derivative is Eq. (31) shifted by (-1/2, -1/2, -1/2): the 8 cells
 * around corner (i, j, k) are (i-1..i, j-1..j, k-1..k).
 */
void ora_div_rhs(int nx, int ny, int nz, double h, double dt, double mu,
                 const double *sig_star, double *b)
{
    long nc = (long)nx * ny * nz;
    /* component index of sigma_ab in the 6-vector xx,yy,zz,yz,xz,xy */
    static const int comp[3][3] = {{0, 5, 4}, {5, 1, 3}, {4, 3, 2}};
    double scale = h * h / (mu * dt) / (4.0 * h);
    memset(b, 0, 3L * (nz + 1) * ny * nx * sizeof(double));
#pragma omp parallel for schedule(static)
    for (int k = 1; k < nz; k++)
        for (int j = 0; j < ny; j++)
            for (int i = 0; i < nx; i++) {
                int im = wrap(i - 1, nx), jm = wrap(j - 1, ny);
                int is[2] = {im, i}, js[2] = {jm, j}, ks[2] = {k - 1, k};
                for (int a = 0; a < 3; a++) {
                    const double *fx = sig_star + comp[a][0] * nc;
                    const double *fy = sig_star + comp[a][1] * nc;
                    const double *fz = sig_star + comp[a][2] * nc;
                    double s = 0.0;
                    for (int u = 0; u < 2; u++)
                        for (int w = 0; w < 2; w++) {
                            s += fx[cell(nx, ny, ks[w], js[u], i)] - fx[cell(nx, ny, ks[w], js[u], im)];
                            s += fy[cell(nx, ny, ks[w], j, is[u])] - fy[cell(nx, ny, ks[w], jm, is[u])];
                            s += fz[cell(nx, ny, k, js[w], is[u])] - fz[cell(nx, ny, k - 1, js[w], is[u])];
                        }
                    b[node(nx, ny, nz, a, k, j, i)] = scale * s;
                }
            }
}

/* stress correction, Eq. (29): sigma = sigma* + dt C:D^{n+1}, D^{n+1} the
 * symmetric part of the Eq. (31) gradient of v^{n+1} */
void ora_stress_final(int nx, int ny, int nz, double h, double dt, double lam, double mu,
                      const double *v, const double *sig_star, double *sig)
{
    long nc = (long)nx * ny * nz;
#pragma omp parallel for schedule(static)
    for (int k = 0; k < nz; k++)
        for (int j = 0; j < ny; j++)
            for (int i = 0; i < nx; i++) {
                long q = cell(nx, ny, k, j, i);
                double L[3][3];
                cell_grad(nx, ny, nz, v, h, k, j, i, L);
                double trD = L[0][0] + L[1][1] + L[2][2];
                sig[0 * nc + q] = sig_star[0 * nc + q] + dt * (lam * trD + 2.0 * mu * L[0][0]);
                sig[1 * nc + q] = sig_star[1 * nc + q] + dt * (lam * trD + 2.0 * mu * L[1][1]);
                sig[2 * nc + q] = sig_star[2 * nc + q] + dt * (lam * trD + 2.0 * mu * L[2][2]);
                sig[3 * nc + q] = sig_star[3 * nc + q] + dt * mu * (L[1][2] + L[2][1]);
                sig[4 * nc + q] = sig_star[4 * nc + q] + dt * mu * (L[0][2] + L[2][0]);
                sig[5 * nc + q] = sig_star[5 * nc + q] + dt * mu * (L[0][1] + L[1][0]);
            }
}

/*
 * Wall velocities at time t on planes k = 0 and k = nz.
 * kind 0, simple shear (Eqs. 37-38): v(z = +-H/2) = (+-U(t), 0, 0),
 *   U = U_B t / t_ramp for t < t_ramp, else U_B.
 * kinds 1-3, spinning disc (section 5, Eqs. 48-49, read as a rotation with
 *   angular velocity omega): u = -omega y f, v = omega x f, w = 0, with
 *   f = 1 for r^2 < R^2 else exp(-lambda_w (r^2 - R^2)^2), r^2 = (x^2+y^2)/L^2,
 *   L the half-width in x; corners sit at x = -L + i h, y = -ny h/2 + j h.
 *   kind 1: top only (bottom fixed); 2: both walls the same; 3: opposite.
 */
void ora_wall_fill(int nx, int ny, int nz, double h, const ora_bc *bc, double t, double *v)
{
    for (int j = 0; j < ny; j++)
        for (int i = 0; i < nx; i++) {
            double top[3] = {0.0, 0.0, 0.0}, bot[3] = {0.0, 0.0, 0.0};
            if (bc->kind == 0) {
                double U = (t < bc->t_ramp) ? bc->U_B * t / bc->t_ramp : bc->U_B;
                top[0] = U;
                bot[0] = -U;
            } else {
                double L = 0.5 * nx * h;
                double x = -L + i * h, y = -0.5 * ny * h + j * h;
                double r2 = (x * x + y * y) / (L * L);
                double R2 = bc->R * bc->R;
                double f = (r2 < R2) ? 1.0 : exp(-bc->lambda_w * (r2 - R2) * (r2 - R2));
                top[0] = -bc->omega * y * f;
                top[1] = bc->omega * x * f;
                double sgn = (bc->kind == 2) ? 1.0 : (bc->kind == 3 ? -1.0 : 0.0);
                bot[0] = sgn * top[0];
                bot[1] = sgn * top[1];
            }
            for (int a = 0; a < 3; a++) {
                v[node(nx, ny, nz, a, 0, j, i)] = bot[a];
                v[node(nx, ny, nz, a, nz, j, i)] = top[a];
            }
        }
}

/*
 * One quasi-static projection step (section 3.3) from time t to t + dt:
 *   1. sigma*, D^pl from (v^n, sigma^n, chi^n)            Eq. (27), (20)-(22)
 *   2. chi^{n+1}                                           Eq. (26)
 *   3. wall velocities at t + dt                           Eqs. (37)-(38)
 *   4. b = (h^2/(mu dt)) div sigma*                        Eq. (30)
 *   5. multigrid solve for v^{n+1}, warm-started from v^n  section 3.6
 *   6. sigma^{n+1} = sigma* + dt C:D^{n+1}                 Eq. (29)
 * Returns the solver status (0 ok, 5 not converged, 6 non-finite).
 */
int ora_qs_step_adv(ora_mg *m, double h, double dt, double lam, double mu, const ora_stz *p,
                    const ora_bc *bc, double t, double *v, double *sig, double *chi, double tol,
                    int max_cycles, int *cycles, double *hist, int advect)
{
    int nx = m->dims[0][0], ny = m->dims[0][1], nz = m->dims[0][2];
    long nc = (long)nx * ny * nz, nn = 3L * (nz + 1) * ny * nx;
    double *sig_star = (double *)malloc(6 * nc * sizeof(double));
    double *dpl = (double *)malloc(nc * sizeof(double));
    double *sbar = (double *)malloc(nc * sizeof(double));
    double *chi_new = (double *)malloc(nc * sizeof(double));
    double *b = (double *)malloc(nn * sizeof(double));
    ora_stress_star_adv(nx, ny, nz, h, dt, mu, p, v, sig, chi, sig_star, dpl, sbar, advect);
    ora_chi_update(nx, ny, nz, h, dt, p, sig, chi, dpl, sbar, chi_new);
    memcpy(chi, chi_new, nc * sizeof(double));
    ora_wall_fill(nx, ny, nz, h, bc, t + dt, v);
    ora_div_rhs(nx, ny, nz, h, dt, mu, sig_star, b);
    int st = ora_mg_solve(m, b, v, tol, max_cycles, cycles, hist);
    ora_stress_final(nx, ny, nz, h, dt, lam, mu, v, sig_star, sig);
    free(sig_star);
    free(dpl);
    free(sbar);
    free(chi_new);
    free(b);
    return st;
}

int ora_qs_step(ora_mg *m, double h, double dt, double lam, double mu, const ora_stz *p,
                const ora_bc *bc, double t, double *v, double *sig, double *chi, double tol,
                int max_cycles, int *cycles, double *hist)
{
    return ora_qs_step_adv(m, h, dt, lam, mu, p, bc, t, v, sig, chi, tol, max_cycles, cycles,
                           hist, 0);
}

/* ------------------------------------------------------------------ */
/* explicit method (section 3.2, Eqs. 24-26; ENO advection, Eq. 33)    */
/* ------------------------------------------------------------------ */

/*
 * ENO first derivative along one line, Eq. (33): f[0..4] are the values at
 * offsets -2..2 (spacing h) around the point and u the velocity component
 * along the line there.  The one-sided three-point derivative on the
 * upwind side is taken when the second derivative (Eq. 32) at the point
 * exceeds in magnitude the one at the upwind neighbour; otherwise the
 * centred difference.
 */
double ora_eno(const double *f, double u, double h)
{
    double fxx_m = (f[2] - 2.0 * f[1] + f[0]) / (h * h);
    double fxx_0 = (f[3] - 2.0 * f[2] + f[1]) / (h * h);
    double fxx_p = (f[4] - 2.0 * f[3] + f[2]) / (h * h);
    if (u < 0.0 && fabs(fxx_0) > fabs(fxx_p))
        return (-f[4] + 4.0 * f[3] - 3.0 * f[2]) / (2.0 * h);
    if (u > 0.0 && fabs(fxx_0) > fabs(fxx_m))
        return (3.0 * f[2] - 4.0 * f[1] + f[0]) / (2.0 * h);
    return (f[3] - f[1]) / (2.0 * h);
}

/* corner value of component a at plane kk, which may lie up to two planes
 * beyond a wall: there the field is reflected through the wall value
 * (Dirichlet ghost, section 3.5): v(-m) = 2 v(0) - v(m) */
static double corner_val(const double *v, int nx, int ny, int nz, int a, int kk, int j, int i)
{
    if (kk < 0)
        return 2.0 * v[node(nx, ny, nz, a, 0, j, i)] - v[node(nx, ny, nz, a, -kk, j, i)];
    if (kk > nz)
        return 2.0 * v[node(nx, ny, nz, a, nz, j, i)] - v[node(nx, ny, nz, a, 2 * nz - kk, j, i)];
    return v[node(nx, ny, nz, a, kk, j, i)];
}

/* cell value of the scalar field f at layer kk, which may lie up to two
 * layers beyond the z boundary: there the field is extrapolated linearly
 * from the two nearest layers (free boundary ghost, section 3.5) */
static double cell_val(const double *f, int nx, int ny, int nz, int kk, int j, int i)
{
    if (kk < 0)
        return f[cell(nx, ny, 0, j, i)] + kk * (f[cell(nx, ny, 1, j, i)] - f[cell(nx, ny, 0, j, i)]);
    if (kk > nz - 1)
        return f[cell(nx, ny, nz - 1, j, i)] +
               (kk - (nz - 1)) * (f[cell(nx, ny, nz - 1, j, i)] - f[cell(nx, ny, nz - 2, j, i)]);
    return f[cell(nx, ny, kk, j, i)];
}

/*
 * One explicit forward-Euler step (section 3.2) from t to t + dt, in place,
 * every right-hand side from the state at t:
 *   sigma: Eq. (25), -(u.grad) sigma + L sigma + sigma L^T - tr(L) sigma
 *          + C:(D - D^pl sigma0 / sbar), at cell centres; L and D from the
 *          Eq. (31) gradient of v; u the mean of the cell's 8 corner
 *          velocities; the advection by ENO (Eq. 33) along x, y, z;
 *   chi:   Eq. (26), as in the quasi-static step;
 *   v:     Eq. (24) at interior corners, rho (v' - v)/dt = -rho (v.grad) v
 *          + div sigma + rho kappa lap v, with the corner divergence of
 *          Eq. (31), the Laplacian of Eq. (32) and ENO advection;
 *   walls at t + dt (Eqs. 37-38, 48-49).
 * kappa is the damping diffusivity (m^2/s), kappa = kappa' h in section 4.
 */
void ora_explicit_step(int nx, int ny, int nz, double h, double dt, double rho, double lam,
                       double mu, double kappa, const ora_stz *p, const ora_bc *bc, double t,
                       double *v, double *sig, double *chi)
{
    static const int comp[3][3] = {{0, 5, 4}, {5, 1, 3}, {4, 3, 2}};
    long nc = (long)nx * ny * nz, nn = 3L * (nz + 1) * ny * nx;
    double *v0 = (double *)malloc(nn * sizeof(double));
    double *s0 = (double *)malloc(6 * nc * sizeof(double));
    double *dpl = (double *)malloc(nc * sizeof(double));
    double *sbar = (double *)malloc(nc * sizeof(double));
    double *chi_new = (double *)malloc(nc * sizeof(double));
    memcpy(v0, v, nn * sizeof(double));
    memcpy(s0, sig, 6 * nc * sizeof(double));

    /* stress, Eq. (25) */
#pragma omp parallel for schedule(static)
    for (int k = 0; k < nz; k++)
        for (int j = 0; j < ny; j++)
            for (int i = 0; i < nx; i++) {
                long q = cell(nx, ny, k, j, i);
                double s6[6], s[3][3], L[3][3], u[3] = {0.0, 0.0, 0.0};
                for (int c = 0; c < 6; c++)
                    s6[c] = s0[c * nc + q];
                sym_full(s6, s);
                cell_grad(nx, ny, nz, v0, h, k, j, i, L);
                for (int a = 0; a < 3; a++)
                    for (int dk = 0; dk < 2; dk++)
                        for (int dj = 0; dj < 2; dj++)
                            for (int di = 0; di < 2; di++)
                                u[a] += 0.125 * v0[node(nx, ny, nz, a, k + dk, wrap(j + dj, ny),
                                                        wrap(i + di, nx))];
                double sb = sbar_of(s);
                double D = ora_dpl(p, sb, chi[q]);
                dpl[q] = D;
                sbar[q] = sb;
                double adv[6];
                for (int c = 0; c < 6; c++) {
                    const double *f = s0 + c * nc;
                    double fx[5], fy[5], fz[5];
                    for (int m = -2; m <= 2; m++) {
                        fx[m + 2] = f[cell(nx, ny, k, j, wrap(i + m, nx))];
                        fy[m + 2] = f[cell(nx, ny, k, wrap(j + m, ny), i)];
                        fz[m + 2] = cell_val(f, nx, ny, nz, k + m, j, i);
                    }
                    adv[c] = u[0] * ora_eno(fx, u[0], h) + u[1] * ora_eno(fy, u[1], h) +
                             u[2] * ora_eno(fz, u[2], h);
                }
                double trL = L[0][0] + L[1][1] + L[2][2];
                double tr3 = (s[0][0] + s[1][1] + s[2][2]) / 3.0;
                double rate[3][3];
                for (int a = 0; a < 3; a++)
                    for (int b = 0; b < 3; b++) {
                        double r = -adv[comp[a][b]] - trL * s[a][b];
                        for (int c = 0; c < 3; c++)
                            r += L[a][c] * s[c][b] + s[a][c] * L[b][c];
                        /* C:D with D = (L + L^T)/2 */
                        r += (a == b ? lam * trL : 0.0) + mu * (L[a][b] + L[b][a]);
                        if (D > 0.0)
                            r -= 2.0 * mu * D * (s[a][b] - (a == b ? tr3 : 0.0)) / sb;
                        rate[a][b] = r;
                    }
                sig[0 * nc + q] = s[0][0] + dt * rate[0][0];
                sig[1 * nc + q] = s[1][1] + dt * rate[1][1];
                sig[2 * nc + q] = s[2][2] + dt * rate[2][2];
                sig[3 * nc + q] = s[1][2] + dt * rate[1][2];
                sig[4 * nc + q] = s[0][2] + dt * rate[0][2];
                sig[5 * nc + q] = s[0][1] + dt * rate[0][1];
            }

    /* effective temperature, Eq. (26), from the state at t */
    ora_chi_update(nx, ny, nz, h, dt, p, s0, chi, dpl, sbar, chi_new);
    memcpy(chi, chi_new, nc * sizeof(double));

    /* velocity, Eq. (24), at interior corners */
#pragma omp parallel for schedule(static)
    for (int k = 1; k < nz; k++)
        for (int j = 0; j < ny; j++)
            for (int i = 0; i < nx; i++) {
                int im = wrap(i - 1, nx), jm = wrap(j - 1, ny);
                int is[2] = {im, i}, js[2] = {jm, j}, ks[2] = {k - 1, k};
                double u[3];
                for (int a = 0; a < 3; a++)
                    u[a] = v0[node(nx, ny, nz, a, k, j, i)];
                for (int a = 0; a < 3; a++) {
                    /* corner divergence of sigma (Eq. 31 shifted by -1/2) */
                    const double *fx = s0 + comp[a][0] * nc;
                    const double *fy = s0 + comp[a][1] * nc;
                    const double *fz = s0 + comp[a][2] * nc;
                    double div = 0.0;
                    for (int e = 0; e < 2; e++)
                        for (int w = 0; w < 2; w++) {
                            div += fx[cell(nx, ny, ks[w], js[e], i)] - fx[cell(nx, ny, ks[w], js[e], im)];
                            div += fy[cell(nx, ny, ks[w], j, is[e])] - fy[cell(nx, ny, ks[w], jm, is[e])];
                            div += fz[cell(nx, ny, k, js[w], is[e])] - fz[cell(nx, ny, k - 1, js[w], is[e])];
                        }
                    div /= 4.0 * h;
                    /* Laplacian, Eq. (32) in x, y and z */
                    double c0 = u[a];
                    double lap = (v0[node(nx, ny, nz, a, k, j, wrap(i + 1, nx))] - 2.0 * c0 +
                                  v0[node(nx, ny, nz, a, k, j, im)]) +
                                 (v0[node(nx, ny, nz, a, k, wrap(j + 1, ny), i)] - 2.0 * c0 +
                                  v0[node(nx, ny, nz, a, k, jm, i)]) +
                                 (v0[node(nx, ny, nz, a, k + 1, j, i)] - 2.0 * c0 +
                                  v0[node(nx, ny, nz, a, k - 1, j, i)]);
                    lap /= h * h;
                    /* ENO advection (Eq. 33) */
                    double fxl[5], fyl[5], fzl[5];
                    for (int m = -2; m <= 2; m++) {
                        fxl[m + 2] = v0[node(nx, ny, nz, a, k, j, wrap(i + m, nx))];
                        fyl[m + 2] = v0[node(nx, ny, nz, a, k, wrap(j + m, ny), i)];
                        fzl[m + 2] = corner_val(v0, nx, ny, nz, a, k + m, j, i);
                    }
                    double adv = u[0] * ora_eno(fxl, u[0], h) + u[1] * ora_eno(fyl, u[1], h) +
                                 u[2] * ora_eno(fzl, u[2], h);
                    v[node(nx, ny, nz, a, k, j, i)] = c0 + dt * (-adv + div / rho + kappa * lap);
                }
            }
    ora_wall_fill(nx, ny, nz, h, bc, t + dt, v);
    free(v0);
    free(s0);
    free(dpl);
    free(sbar);
    free(chi_new);
}

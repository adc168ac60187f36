// mg_kernels.cu -- multigrid kernels for the scaled projection operator
// (Eq. 30 discretised with the stencils of section 3.4; V-cycle of section 3.6).
//
// Layout: corner arrays (3, nz+1, ny, nx), x fastest; planes 0 and nz hold the
// Dirichlet walls (zero on coarse levels); x and y wrap periodically.
// Colour of node (i, j, k): (i&1) + 2(j&1) + 4(k&1); a colour pass updates all
// nodes of one colour at once (no two of them are coupled: every stencil
// offset lies in {-1,0,1}^3 and the sizes are even).
#include "qsmg_impl.h"

namespace qsmg {
namespace {

constexpr int kThreads = 256;

inline unsigned nblocks(long n, int t = kThreads) { return (unsigned)((n + t - 1) / t); }

// ---------------------------------------------------------------------------
// finest-level operator (structured 19-point stencil)
// ---------------------------------------------------------------------------

// column position of x index i in a row: natural, or parity-split (the even
// nodes of the row first, then the odd ones; used for the finest FP32 arrays)
__device__ __forceinline__ int colmap(int i, int nx, int split) {
    return split ? ((i & 1) * (nx >> 1) + (i >> 1)) : i;
}

// value of x at plane kk; with WO ("walls only") interior planes read as zero
template <typename T, bool WO>
__device__ __forceinline__ T ldx(const T *x, long idx, int kk, int nz) {
    if (WO && kk > 0 && kk < nz) return T(0);
    return x[idx];
}

// o_a = sum over the 18 non-centre offsets of S_d[a][b] x_b(p + d)
//   = -( lp x_a(+-e_a) + x_a(+-e_b, b != a) + kq sum_{b!=a} M_ab[x_b] ),
// M_ab[g] = g(+a,+b) - g(+a,-b) - g(-a,+b) + g(-a,-b)  (4-point mixed difference)
template <typename T, bool WO>
__device__ __forceinline__ void fine_off(const T *x, const Dims &d, int i0, int j, int k, T lp,
                                         T kq, T o[3], int split = 0) {
    const int nx = d.nx, ny = d.ny, nz = d.nz;
    const long ps = (long)nx * ny;
    const int im = colmap(i0 ? i0 - 1 : nx - 1, nx, split),
              ip = colmap((i0 + 1 < nx) ? i0 + 1 : 0, nx, split);
    const int i = colmap(i0, nx, split);
    const int jm = j ? j - 1 : ny - 1, jp = (j + 1 < ny) ? j + 1 : 0;
    const long pc = (long)k * ps, pm = pc - ps, pp = pc + ps;
    const long r0 = (long)j * nx, rm = (long)jm * nx, rp = (long)jp * nx;
    const T *x0 = x, *x1 = x + d.cs, *x2 = x + 2 * d.cs;
#define XC(g, r, c) ldx<T, WO>(g, pc + (r) + (c), k, nz)
#define XM(g, r, c) ldx<T, WO>(g, pm + (r) + (c), k - 1, nz)
#define XP(g, r, c) ldx<T, WO>(g, pp + (r) + (c), k + 1, nz)
    const T a0 = lp * (XC(x0, r0, im) + XC(x0, r0, ip)) + (XC(x0, rm, i) + XC(x0, rp, i)) +
                 (XM(x0, r0, i) + XP(x0, r0, i));
    const T a1 = lp * (XC(x1, rm, i) + XC(x1, rp, i)) + (XC(x1, r0, im) + XC(x1, r0, ip)) +
                 (XM(x1, r0, i) + XP(x1, r0, i));
    const T a2 = lp * (XM(x2, r0, i) + XP(x2, r0, i)) + (XC(x2, r0, im) + XC(x2, r0, ip)) +
                 (XC(x2, rm, i) + XC(x2, rp, i));
#define MXY(g) (XC(g, rp, ip) - XC(g, rm, ip) - XC(g, rp, im) + XC(g, rm, im))
#define MXZ(g) (XP(g, r0, ip) - XM(g, r0, ip) - XP(g, r0, im) + XM(g, r0, im))
#define MYZ(g) (XP(g, rp, i) - XM(g, rp, i) - XP(g, rm, i) + XM(g, rm, i))
    o[0] = -(a0 + kq * (MXY(x1) + MXZ(x2)));
    o[1] = -(a1 + kq * (MXY(x0) + MYZ(x2)));
    o[2] = -(a2 + kq * (MXZ(x0) + MYZ(x1)));
#undef XC
#undef XM
#undef XP
#undef MXY
#undef MXZ
#undef MYZ
}

// coarse 27-point block stencil, off-centre part, in parity-class form
template <typename T>
__device__ __forceinline__ void coarse_off(const T *x, const Dims &d, int i, int j, int k,
                                           const Coarse<T> &c, T o[3]) {
    const int nx = d.nx, ny = d.ny;
    const long ps = (long)nx * ny;
    const int im = i ? i - 1 : nx - 1, ip = i + 1 < nx ? i + 1 : 0;
    const int jm = j ? j - 1 : ny - 1, jp = j + 1 < ny ? j + 1 : 0;
    const int col[3] = {im, i, ip};
    const long row[3] = {(long)jm * nx, (long)j * nx, (long)jp * nx};
    const long pc = (long)k * ps;
    auto u = [&](int b, int dx, int dy) -> T {
        return x[b * d.cs + pc + row[dy + 1] + col[dx + 1]];
    };
    auto sd = [&](int b, int dx, int dy, T &S, T &D) {
        const long q = b * d.cs + pc + row[dy + 1] + col[dx + 1];
        const T lo = x[q - ps], hi = x[q + ps];
        S = hi + lo;
        D = hi - lo;
    };
    coarse_plane_terms(c, u, o);
    coarse_z_terms(c, sd, o);
}

// launch shape of the node kernels: 32 x 8 threads over (i, j), grid.z over
// planes, so no thread divides a flat index
constexpr int BX = 32, BY = 8;

// node of colour `colour` handled by this thread (false if outside)
__device__ __forceinline__ bool colour_node(int colour, int hx, int hy, int &i, int &j, int &k) {
    const int ix = blockIdx.x * BX + threadIdx.x, jy = blockIdx.y * BY + threadIdx.y;
    if (ix >= hx || jy >= hy) return false;
    i = 2 * ix + (colour & 1);
    j = 2 * jy + ((colour >> 1) & 1);
    k = 2 * (int)blockIdx.z + ((colour & 4) ? 1 : 2);
    return true;
}

// interior node (i, j, k), k in 1..nz-1, handled by this thread
__device__ __forceinline__ bool node_ijk(const Dims &d, int &i, int &j, int &k) {
    i = blockIdx.x * BX + threadIdx.x;
    j = blockIdx.y * BY + threadIdx.y;
    k = blockIdx.z + 1;
    return i < d.nx && j < d.ny;
}

// planes of one k-parity among the interior planes 1..nz-1
inline int colour_planes(int nz, int colour) { return (colour & 4) ? nz / 2 : nz / 2 - 1; }

template <typename T>
__global__ void k_gs_fine(Dims d, Fine<T> f, const T *__restrict__ b, T *x, int colour, int hx,
                          int hy) {
    int i, j, k;
    if (!colour_node(colour, hx, hy, i, j, k)) return;
    T o[3];
    fine_off<T, false>(x, d, i, j, k, f.lp, f.kq, o);
    const long p = ((long)k * d.ny + j) * d.nx + i;
    const T u0 = (b[p] - o[0]) * f.dinv;
    const T u1 = (b[p + d.cs] - o[1]) * f.dinv;
    const T u2 = (b[p + 2 * d.cs] - o[2]) * f.dinv;
    x[p] = u0;
    x[p + d.cs] = u1;
    x[p + 2 * d.cs] = u2;
}

template <typename T>
__global__ void k_gs_coarse(Dims d, Coarse<T> c, const T *__restrict__ b, T *x, int colour, int hx,
                            int hy) {
    int i, j, k;
    if (!colour_node(colour, hx, hy, i, j, k)) return;
    T o[3];
    coarse_off<T>(x, d, i, j, k, c, o);
    const long p = ((long)k * d.ny + j) * d.nx + i;
#pragma unroll
    for (int a = 0; a < 3; a++) x[p + a * d.cs] = c.dinv[a] * (b[p + a * d.cs] - o[a]);
}

template <typename T>
__global__ void k_res_fine(Dims d, Fine<T> f, const T *__restrict__ b, const T *__restrict__ x,
                           T *__restrict__ r, int split) {
    int i, j, k;
    if (!node_ijk(d, i, j, k)) return;
    T o[3];
    fine_off<T, false>(x, d, i, j, k, f.lp, f.kq, o, split);
    const long p = ((long)k * d.ny + j) * d.nx + colmap(i, d.nx, split);
#pragma unroll
    for (int a = 0; a < 3; a++) r[p + a * d.cs] = b[p + a * d.cs] - (f.d0 * x[p + a * d.cs] + o[a]);
}

template <typename T>
__global__ void k_res_coarse(Dims d, Coarse<T> c, const T *__restrict__ b,
                             const T *__restrict__ x, T *__restrict__ r) {
    int i, j, k;
    if (!node_ijk(d, i, j, k)) return;
    T o[3];
    coarse_off<T>(x, d, i, j, k, c, o);
    const long p = ((long)k * d.ny + j) * d.nx + i;
#pragma unroll
    for (int a = 0; a < 3; a++)
        r[p + a * d.cs] = b[p + a * d.cs] - (o[a] + c.cd[a][0] * x[p + a * d.cs]);
}

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    return v;
}

// fixed-order block sum; result valid in thread 0
__device__ double block_sum(double v) {
    __shared__ double sh[32];
    v = warp_sum(v);
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    __syncthreads();
    if (l == 0) sh[w] = v;
    __syncthreads();
    const int nw = blockDim.x >> 5;
    v = (threadIdx.x < (unsigned)nw) ? sh[threadIdx.x] : 0.0;
    if (w == 0) v = warp_sum(v);
    return v;
}

template <bool WO>
__global__ void __launch_bounds__(kRedThreads)
    k_res_norm_fine64(Dims d, Fine<double> f, const double *__restrict__ b,
                      const double *__restrict__ x, float *__restrict__ r32, double out_scale,
                      double *__restrict__ partials, int split32) {
    // rows (j, k) are dealt to blocks in a fixed order, columns to threads,
    // so the partial sums do not depend on timing
    double acc = 0.0;
    const int nrows = d.ny * (d.nz - 1);
    for (int row = blockIdx.x; row < nrows; row += gridDim.x) {
        const int k = row / d.ny + 1, j = row - (k - 1) * d.ny;
        if (WO && k != 1 && k != d.nz - 1) {
            // away from the walls the lifted right-hand side is b itself
            const long p0 = ((long)k * d.ny + j) * d.nx;
            for (int i = threadIdx.x; i < d.nx; i += blockDim.x)
#pragma unroll
                for (int a = 0; a < 3; a++) {
                    const double r = b[p0 + i + a * d.cs];
                    acc += r * r;
                }
            continue;
        }
        for (int i = threadIdx.x; i < d.nx; i += blockDim.x) {
            double o[3];
            fine_off<double, WO>(x, d, i, j, k, f.lp, f.kq, o);
            const long p = ((long)k * d.ny + j) * d.nx + i;
#pragma unroll
            for (int a = 0; a < 3; a++) {
                const double xc = WO ? 0.0 : x[p + a * d.cs];
                const double r = b[p + a * d.cs] - (f.d0 * xc + o[a]);
                acc += r * r;
                if (r32) r32[p - i + colmap(i, d.nx, split32) + a * d.cs] = (float)(r * out_scale);
            }
        }
    }
    const double s = block_sum(acc);
    if (threadIdx.x == 0) partials[blockIdx.x] = s;
}

__global__ void __launch_bounds__(kRedThreads)
    k_sumsq(Dims d, const double *__restrict__ r, double *__restrict__ partials) {
    double acc = 0.0;
    const int nrows = d.ny * (d.nz - 1);
    for (int row = blockIdx.x; row < nrows; row += gridDim.x) {
        const long p0 = (long)(row + d.ny) * d.nx;  // interior rows start at plane 1
        for (int i = threadIdx.x; i < d.nx; i += blockDim.x)
#pragma unroll
            for (int a = 0; a < 3; a++) {
                const double v = r[p0 + i + a * d.cs];
                acc += v * v;
            }
    }
    const double s = block_sum(acc);
    if (threadIdx.x == 0) partials[blockIdx.x] = s;
}

__global__ void __launch_bounds__(1024) k_sum_partials(const double *__restrict__ partials,
                                                        double *__restrict__ out) {
    double acc = 0.0;
    for (int t = threadIdx.x; t < kRedBlocks; t += 1024) acc += partials[t];
    const double s = block_sum(acc);
    if (threadIdx.x == 0) out[0] = s;
}

// restriction R = T^T (full weighting, weights 1, 1/2, 1/4, 1/8 by the
// number of odd offsets), coarse interior nodes
template <typename T>
__global__ void k_restrict(Dims f, Dims c, const T *__restrict__ r, T *__restrict__ bc,
                           int split) {
    int I, J, K;
    if (!node_ijk(c, I, J, K)) return;
    T s0 = 0, s1 = 0, s2 = 0;
#pragma unroll
    for (int ez = -1; ez <= 1; ez++) {
        const T wz = ez ? T(0.5) : T(1);
        const long pl = (long)(2 * K + ez) * f.ny;
#pragma unroll
        for (int ey = -1; ey <= 1; ey++) {
            const T wy = ey ? T(0.5) : T(1);
            int jj = 2 * J + ey;
            jj = jj < 0 ? jj + f.ny : (jj >= f.ny ? jj - f.ny : jj);
            const long row = (pl + jj) * f.nx;
#pragma unroll
            for (int ex = -1; ex <= 1; ex++) {
                const T w = (ex ? T(0.5) : T(1)) * wy * wz;
                int ii = 2 * I + ex;
                ii = ii < 0 ? ii + f.nx : (ii >= f.nx ? ii - f.nx : ii);
                const long q = row + colmap(ii, f.nx, split);
                s0 += w * r[q];
                s1 += w * r[q + f.cs];
                s2 += w * r[q + 2 * f.cs];
            }
        }
    }
    const long p = ((long)K * c.ny + J) * c.nx + I;
    bc[p] = s0;
    bc[p + c.cs] = s1;
    bc[p + 2 * c.cs] = s2;
}

// z part of the full weighting, after the fused fine residual of
// smoother_rows.cu has applied the x and y parts: bc(I, J, K) = 1/2 p(2K-1)
// + p(2K) + 1/2 p(2K+1), p(k) the partial sums of fine plane k, laid out
// [c][k][J][I] with component stride pcs; coarse interior nodes
__global__ void k_restrict_z(Dims c, long pcs, const float *__restrict__ p,
                             float *__restrict__ bc) {
    int I, J, K;
    if (!node_ijk(c, I, J, K)) return;
    const long pl = (long)c.ny * c.nx, q = (long)J * c.nx + I;
#pragma unroll
    for (int a = 0; a < 3; a++) {
        const float *pa = p + a * pcs + q;
        bc[a * c.cs + K * pl + q] =
            (0.5f * pa[(2 * K - 1) * pl] + pa[2 * K * pl]) + 0.5f * pa[(2 * K + 1) * pl];
    }
}

// prolongation x += T xc: fine node 2I is coarse node I, odd fine nodes take
// the mean of their two neighbours along each odd axis (coarse walls are 0).
// One thread per coarse cell (I, J, K): it loads the cell's 8 corners once
// per component, interpolates separably (x, then y, then z) and adds into
// its 2 x 2 x 2 block of fine nodes (2I+a, 2J+b, 2K+c), wall plane 0 skipped.
template <typename T>
__global__ void k_prolong(Dims f, Dims c, const T *__restrict__ xc, T *__restrict__ x, int split) {
    const int I = blockIdx.x * BX + threadIdx.x, J = blockIdx.y * BY + threadIdx.y;
    const int K = blockIdx.z;
    if (I >= c.nx || J >= c.ny) return;
    const int I1 = I + 1 < c.nx ? I + 1 : 0, J1 = J + 1 < c.ny ? J + 1 : 0;
    const long cps = (long)c.nx * c.ny, fps = (long)f.nx * f.ny;
    const long cr[2] = {(long)J * c.nx, (long)J1 * c.nx};
    const int ci[2] = {I, I1};
    const int fcol[2] = {colmap(2 * I, f.nx, split), colmap(2 * I + 1, f.nx, split)};
    const T h = T(0.5);
    T w[3][2][2][2];  // [component][coarse z][fine b][fine a]
#pragma unroll
    for (int a = 0; a < 3; a++) {
        const T *X = xc + a * c.cs + (long)K * cps;
        T v[2][2][2];  // [z][y][x] corners
#pragma unroll
        for (int z = 0; z < 2; z++)
#pragma unroll
            for (int y = 0; y < 2; y++)
#pragma unroll
                for (int e = 0; e < 2; e++) v[z][y][e] = X[z * cps + cr[y] + ci[e]];
#pragma unroll
        for (int z = 0; z < 2; z++) {
            T ax[2][2];  // [y][fine a]
#pragma unroll
            for (int y = 0; y < 2; y++) {
                ax[y][0] = v[z][y][0];
                ax[y][1] = h * (v[z][y][0] + v[z][y][1]);
            }
#pragma unroll
            for (int e = 0; e < 2; e++) {
                w[a][z][0][e] = ax[0][e];
                w[a][z][1][e] = h * (ax[0][e] + ax[1][e]);
            }
        }
    }
    // every fine value of the block is loaded before any is stored: as far
    // as the compiler knows a store may alias a later load, so interleaved
    // read-modify-writes would wait for one DRAM round trip each
    const int cz0 = K == 0 ? 1 : 0;  // fine plane 0 is a wall
    T old[3][2][2][2];
#pragma unroll
    for (int a = 0; a < 3; a++)
#pragma unroll
        for (int cz = 0; cz < 2; cz++) {
            if (cz < cz0) continue;
#pragma unroll
            for (int bb = 0; bb < 2; bb++) {
                const T *row = x + a * f.cs + (long)(2 * K + cz) * fps + (long)(2 * J + bb) * f.nx;
#pragma unroll
                for (int e = 0; e < 2; e++) old[a][cz][bb][e] = row[fcol[e]];
            }
        }
#pragma unroll
    for (int a = 0; a < 3; a++)
#pragma unroll
        for (int cz = 0; cz < 2; cz++) {
            if (cz < cz0) continue;
#pragma unroll
            for (int bb = 0; bb < 2; bb++) {
                T *row = x + a * f.cs + (long)(2 * K + cz) * fps + (long)(2 * J + bb) * f.nx;
#pragma unroll
                for (int e = 0; e < 2; e++) {
                    const T val = cz ? h * (w[a][0][bb][e] + w[a][1][bb][e]) : w[a][0][bb][e];
                    row[fcol[e]] = old[a][cz][bb][e] + val;
                }
            }
        }
}

// x += Ainv r on the coarsest level; one warp per unknown, fixed-order sums.
// unknown u = (((k-1) ny + j) nx + i) * 3 + a
template <typename T>
__global__ void k_coarse_solve(Dims d, const double *__restrict__ Ainv, int n,
                               const T *__restrict__ r, T *__restrict__ x) {
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (warp >= n) return;
    double acc = 0.0;
    const long plane0 = (long)d.ny * d.nx;
    for (int v = lane; v < n; v += 32) {
        const int a = v % 3;
        const long node = v / 3;  // ((k-1) ny + j) nx + i
        acc += Ainv[(long)warp * n + v] * (double)r[a * d.cs + plane0 + node];
    }
    acc = warp_sum(acc);
    if (lane == 0) {
        const int a = warp % 3;
        const long node = warp / 3;
        const long p = a * d.cs + plane0 + node;
        x[p] = (T)((double)x[p] + acc);
    }
}

__global__ void k_zero_interior(Dims d, double *__restrict__ x) {
    int i, j, k;
    if (!node_ijk(d, i, j, k)) return;
    const long p = ((long)k * d.ny + j) * d.nx + i;
#pragma unroll
    for (int a = 0; a < 3; a++) x[a * d.cs + p] = 0.0;
}

__global__ void k_axpy_f32(Dims d, double scale, const float *__restrict__ e,
                           double *__restrict__ v, int split) {
    int i, j, k;
    if (!node_ijk(d, i, j, k)) return;
    const long row = ((long)k * d.ny + j) * d.nx;
    const long p = row + i, pe = row + colmap(i, d.nx, split);
    // all loads before the stores (a store may alias a later load as far as
    // the compiler knows, which would serialise the three round trips)
    double vo[3];
    float eo[3];
#pragma unroll
    for (int a = 0; a < 3; a++) {
        vo[a] = v[a * d.cs + p];
        eo[a] = e[a * d.cs + pe];
    }
#pragma unroll
    for (int a = 0; a < 3; a++) v[a * d.cs + p] = vo[a] + scale * (double)eo[a];
}

// natural <-> parity-split column order of a whole corner array
template <bool TO_SPLIT>
__global__ void k_split(Dims d, const float *__restrict__ src, float *__restrict__ dst) {
    const int i = blockIdx.x * BX + threadIdx.x, j = blockIdx.y * BY + threadIdx.y;
    const int kc = blockIdx.z;  // component * (nz+1) + plane
    if (i >= d.nx || j >= d.ny) return;
    const long row = ((long)kc * d.ny + j) * d.nx;
    const long a = row + i, b = row + colmap(i, d.nx, 1);
    if (TO_SPLIT) dst[b] = src[a];
    else dst[a] = src[b];
}

inline dim3 node_grid(int nx, int ny, int nplanes) {
    return dim3((nx + BX - 1) / BX, (ny + BY - 1) / BY, nplanes);
}
const dim3 kBlock(BX, BY);

template <typename T>
cudaError_t gs_fine_t(const Dims &d, const Fine<T> &f, const T *b, T *x, int colour,
                      cudaStream_t s) {
    const int hx = d.nx / 2, hy = d.ny / 2, nk = colour_planes(d.nz, colour);
    if (nk <= 0) return cudaSuccess;
    k_gs_fine<T><<<node_grid(hx, hy, nk), kBlock, 0, s>>>(d, f, b, x, colour, hx, hy);
    count_launch();
    return cudaGetLastError();
}

template <typename T>
cudaError_t gs_coarse_t(const Dims &d, const Coarse<T> &c, const T *b, T *x, int colour,
                        cudaStream_t s) {
    const int hx = d.nx / 2, hy = d.ny / 2, nk = colour_planes(d.nz, colour);
    if (nk <= 0) return cudaSuccess;
    k_gs_coarse<T><<<node_grid(hx, hy, nk), kBlock, 0, s>>>(d, c, b, x, colour, hx, hy);
    count_launch();
    return cudaGetLastError();
}

}  // namespace

cudaError_t gs_colour_fine(const Dims &d, const Fine<double> &f, const double *b, double *x,
                           int colour, cudaStream_t s) {
    return gs_fine_t(d, f, b, x, colour, s);
}
cudaError_t gs_colour_fine(const Dims &d, const Fine<float> &f, const float *b, float *x,
                           int colour, cudaStream_t s) {
    return gs_fine_t(d, f, b, x, colour, s);
}
cudaError_t gs_colour_coarse(const Dims &d, const Coarse<double> &c, const double *b, double *x,
                             int colour, cudaStream_t s) {
    return gs_coarse_t(d, c, b, x, colour, s);
}
cudaError_t gs_colour_coarse(const Dims &d, const Coarse<float> &c, const float *b, float *x,
                             int colour, cudaStream_t s) {
    return gs_coarse_t(d, c, b, x, colour, s);
}

template <typename T>
static cudaError_t res_fine_t(const Dims &d, const Fine<T> &f, const T *b, const T *x, T *r,
                              cudaStream_t s, int split) {
    k_res_fine<T><<<node_grid(d.nx, d.ny, d.nz - 1), kBlock, 0, s>>>(d, f, b, x, r, split);
    count_launch();
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    // wall planes of r are zero
    const long plane = (long)d.ny * d.nx;
    for (int a = 0; a < 3; a++) {
        e = cudaMemsetAsync(r + a * d.cs, 0, plane * sizeof(T), s);
        if (e != cudaSuccess) return e;
        e = cudaMemsetAsync(r + a * d.cs + (long)d.nz * plane, 0, plane * sizeof(T), s);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

template <typename T>
static cudaError_t res_coarse_t(const Dims &d, const Coarse<T> &c, const T *b, const T *x, T *r,
                                cudaStream_t s) {
    k_res_coarse<T><<<node_grid(d.nx, d.ny, d.nz - 1), kBlock, 0, s>>>(d, c, b, x, r);
    count_launch();
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    const long plane = (long)d.ny * d.nx;
    for (int a = 0; a < 3; a++) {
        e = cudaMemsetAsync(r + a * d.cs, 0, plane * sizeof(T), s);
        if (e != cudaSuccess) return e;
        e = cudaMemsetAsync(r + a * d.cs + (long)d.nz * plane, 0, plane * sizeof(T), s);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

cudaError_t residual_fine(const Dims &d, const Fine<double> &f, const double *b, const double *x,
                          double *r, cudaStream_t s) {
    return res_fine_t(d, f, b, x, r, s, 0);
}
cudaError_t residual_fine(const Dims &d, const Fine<float> &f, const float *b, const float *x,
                          float *r, cudaStream_t s, int split) {
    // whole-row strips where the rows fit (smoother_rows.cu), else one
    // thread per node
    cudaError_t e = residual_fine_rows(d, f, b, x, r, s, split);
    if (e == cudaErrorNotSupported) return res_fine_t(d, f, b, x, r, s, split);
    if (e != cudaSuccess) return e;
    const long plane = (long)d.ny * d.nx;  // wall planes of r are zero
    for (int a = 0; a < 3; a++) {
        e = cudaMemsetAsync(r + a * d.cs, 0, plane * sizeof(float), s);
        if (e != cudaSuccess) return e;
        e = cudaMemsetAsync(r + a * d.cs + (long)d.nz * plane, 0, plane * sizeof(float), s);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}
cudaError_t residual_coarse(const Dims &d, const Coarse<double> &c, const double *b,
                            const double *x, double *r, cudaStream_t s) {
    return res_coarse_t(d, c, b, x, r, s);
}
cudaError_t residual_coarse(const Dims &d, const Coarse<float> &c, const float *b, const float *x,
                            float *r, cudaStream_t s) {
    return res_coarse_t(d, c, b, x, r, s);
}

cudaError_t residual_norm_fine64(const Dims &d, const Fine<double> &f, const double *b,
                                 const double *x, bool wall_only, float *r32, double out_scale,
                                 double *partials, cudaStream_t s, int split32) {
    if (wall_only)
        k_res_norm_fine64<true><<<kRedBlocks, kRedThreads, 0, s>>>(d, f, b, x, r32, out_scale,
                                                                   partials, split32);
    else
        k_res_norm_fine64<false><<<kRedBlocks, kRedThreads, 0, s>>>(d, f, b, x, r32, out_scale,
                                                                    partials, split32);
    count_launch();
    return cudaGetLastError();
}

cudaError_t sumsq(const Dims &d, const double *r, double *partials, cudaStream_t s) {
    k_sumsq<<<kRedBlocks, kRedThreads, 0, s>>>(d, r, partials);
    count_launch();
    return cudaGetLastError();
}

cudaError_t sum_partials(const double *partials, double *out, cudaStream_t s) {
    k_sum_partials<<<1, 1024, 0, s>>>(partials, out);
    count_launch();
    return cudaGetLastError();
}

template <typename T>
static cudaError_t restrict_t(const Dims &f, const T *r, T *bc, cudaStream_t s, int split) {
    const Dims c = make_dims(f.nx / 2, f.ny / 2, f.nz / 2);
    if (c.nz < 2) return cudaSuccess;
    k_restrict<T><<<node_grid(c.nx, c.ny, c.nz - 1), kBlock, 0, s>>>(f, c, r, bc, split);
    count_launch();
    return cudaGetLastError();
}
cudaError_t restrict_fw(const Dims &fine, const double *r, double *bc, cudaStream_t s) {
    return restrict_t(fine, r, bc, s, 0);
}
cudaError_t restrict_fw(const Dims &fine, const float *r, float *bc, cudaStream_t s, int split) {
    return restrict_t(fine, r, bc, s, split);
}

cudaError_t restrict_z(const Dims &fine, const float *part, float *bc, cudaStream_t s) {
    const Dims c = make_dims(fine.nx / 2, fine.ny / 2, fine.nz / 2);
    if (c.nz < 2) return cudaSuccess;
    const long pcs = (long)(fine.nz + 1) * c.ny * c.nx;
    k_restrict_z<<<node_grid(c.nx, c.ny, c.nz - 1), kBlock, 0, s>>>(c, pcs, part, bc);
    count_launch();
    return cudaGetLastError();
}

template <typename T>
static cudaError_t prolong_t(const Dims &f, const T *xc, T *x, cudaStream_t s, int split) {
    const Dims c = make_dims(f.nx / 2, f.ny / 2, f.nz / 2);
    k_prolong<T><<<node_grid(c.nx, c.ny, c.nz), kBlock, 0, s>>>(f, c, xc, x, split);
    count_launch();
    return cudaGetLastError();
}
cudaError_t prolong_add(const Dims &fine, const double *xc, double *x, cudaStream_t s) {
    return prolong_t(fine, xc, x, s, 0);
}
cudaError_t prolong_add(const Dims &fine, const float *xc, float *x, cudaStream_t s, int split) {
    return prolong_t(fine, xc, x, s, split);
}

template <typename T>
static cudaError_t coarse_t(const Dims &d, const double *Ainv, int n, const T *r, T *x,
                            cudaStream_t s) {
    const long threads = (long)n * 32;
    k_coarse_solve<T><<<nblocks(threads), kThreads, 0, s>>>(d, Ainv, n, r, x);
    count_launch();
    return cudaGetLastError();
}
cudaError_t coarse_solve(const Dims &d, const double *Ainv, int n, const double *r, double *x,
                         cudaStream_t s) {
    return coarse_t(d, Ainv, n, r, x, s);
}
cudaError_t coarse_solve(const Dims &d, const double *Ainv, int n, const float *r, float *x,
                         cudaStream_t s) {
    return coarse_t(d, Ainv, n, r, x, s);
}

cudaError_t zero_interior(const Dims &d, double *x, cudaStream_t s) {
    k_zero_interior<<<node_grid(d.nx, d.ny, d.nz - 1), kBlock, 0, s>>>(d, x);
    count_launch();
    return cudaGetLastError();
}

cudaError_t axpy_f32(const Dims &d, double scale, const float *e, double *v, cudaStream_t s,
                     int split) {
    k_axpy_f32<<<node_grid(d.nx, d.ny, d.nz - 1), kBlock, 0, s>>>(d, scale, e, v, split);
    count_launch();
    return cudaGetLastError();
}

cudaError_t split_columns(const Dims &d, const float *src, float *dst, bool to_split,
                          cudaStream_t s) {
    const dim3 grid = node_grid(d.nx, d.ny, 3 * (d.nz + 1));
    if (to_split)
        k_split<true><<<grid, kBlock, 0, s>>>(d, src, dst);
    else
        k_split<false><<<grid, kBlock, 0, s>>>(d, src, dst);
    count_launch();
    return cudaGetLastError();
}

}  // namespace qsmg

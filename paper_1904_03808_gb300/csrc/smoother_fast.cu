// smoother_fast.cu -- tiled two-phase Gauss-Seidel sweeps (any level).
//
// One 8-colour sweep (colours (i&1)+2(j&1)+4(k&1), visited 0..7, or 7..0)
// in two launches.  Colours 0-3 live on the even-k planes and 4-7 on the
// odd-k planes, and the stencil couples a plane only to its two neighbours,
// so:
//   phase 1 updates every plane of the first k-parity (its 4 in-plane colours
//           in order), reading its z-neighbours' old values;
//   phase 2 updates every plane of the other parity, reading the new values
//           phase 1 wrote.
// This is the same computation as eight colour passes (every node sees the
// same neighbour values), with v read and written about twice per sweep
// instead of eight times.
//
// Which kernel implements a phase (FP32): rows of 64, 128, 192 or 256 nodes
// take the persistent row-strip kernel of smoother_rows.cu (finest level, and
// coarse levels of rows >= 128 nodes), other finest rows of up to 512 nodes
// its per-tile row-strip kernel; coarse planes of at most 32 x 32 nodes take
// the whole-plane kernel further below.  Everything else -- wider finest
// rows, the 64^3-like coarse levels -- takes the tile kernel: inside one
// plane a CTA owns a TX x TY tile and stages a window of that plane
// with a halo of HX columns and HY rows in shared memory (17 KB in FP32); the
// z-neighbour planes and the right-hand side, which the phase only reads,
// come through the read-only cache.  The same kernel
// serves the finest level (structured 19-point operator) and the coarse
// levels (Galerkin 27-point block stencil); both couple a node only to the 8
// in-plane neighbours and to 9 nodes in each adjacent plane.  The 4 in-plane colours are
// computed on shrinking regions so that the tile's own nodes see exactly the
// neighbour values of the sequential order (the halo nodes are recomputed,
// identically, by the neighbouring CTAs).  The sweep is out of place (vin ->
// vout) so no CTA ever reads a value another CTA has already overwritten;
// vout's wall planes must hold the wall values.
#include "qsmg_impl.h"

namespace qsmg {
namespace {

constexpr int TX = 64, TY = 16;        // tile owned by one CTA
constexpr int HX = 4, HY = 2;          // staging halo (x, y)
constexpr int WX = TX + 2 * HX;        // 72 window columns
constexpr int WY = TY + 2 * HY;        // 20 window rows
constexpr int WH = WX / 2;             // words per parity half-row
constexpr int WIN1 = WY * WX;          // one component of a window
constexpr int WIN = 3 * WIN1;          // three components
constexpr int NT = 256;

template <typename T, bool STAGE_Z>
constexpr size_t smem_bytes() {
    return (STAGE_Z ? 3 : 1) * WIN * sizeof(T) + (WX + WY) * sizeof(int);
}

// window element (component c, row wy, column wx): columns split by parity so
// that the 2-strided nodes of one colour sit in consecutive words
__device__ __forceinline__ int widx(int c, int wy, int wx) {
    return ((c * WY + wy) * 2 + (wx & 1)) * WH + (wx >> 1);
}

__device__ __forceinline__ int wrap_mod(int a, int n) {
    a %= n;
    return a < 0 ? a + n : a;
}

// what one node update sees: the staged plane P (shared memory), the
// z-neighbour planes L, H and the right-hand side B of this plane (global,
// read-only), addressed through the wrapped row / column offsets rowg, colg
template <typename T>
struct View {
    T *P;
    const T *__restrict__ L;
    const T *__restrict__ H;
    const T *__restrict__ B;
    long cs;
    const int *rowg, *colg;
    const T *Ls, *Hs;  // staged z-neighbour windows (operators with kStageZ)
};

// finest level: the structured 19-point operator (scaled Eq. 30).  Its
// z-neighbour planes are read through the read-only cache: staging them in
// shared memory as well was measured slower on GB300 (0.50 against 0.36 ms a
// sweep at 256^3), the extra staging traffic outweighing the stride-2 reads
template <typename T>
struct FineOp {
    static constexpr bool kStageZ = false;
    Fine<T> f;
    __device__ __forceinline__ void update(const View<T> &v, int wx, int wy) const {
        T *P = v.P;
        const long cs = v.cs;
        const int xm = wx - 1, xp = wx + 1, ym = wy - 1, yp = wy + 1;
        const int g00 = v.rowg[wy] + v.colg[wx];
        const int gm0 = v.rowg[wy] + v.colg[xm], gp0 = v.rowg[wy] + v.colg[xp];
        const int g0m = v.rowg[ym] + v.colg[wx], g0p = v.rowg[yp] + v.colg[wx];
        const T lp = f.lp, kq = f.kq;
#define Pv(c, yy, xx) P[widx(c, yy, xx)]
#define Lg(c, g) __ldg(v.L + (c) * cs + (g))
#define Hg(c, g) __ldg(v.H + (c) * cs + (g))
        const T a0 = lp * (Pv(0, wy, xm) + Pv(0, wy, xp)) + (Pv(0, ym, wx) + Pv(0, yp, wx)) +
                     (Lg(0, g00) + Hg(0, g00));
        const T a1 = lp * (Pv(1, ym, wx) + Pv(1, yp, wx)) + (Pv(1, wy, xm) + Pv(1, wy, xp)) +
                     (Lg(1, g00) + Hg(1, g00));
        const T a2 = lp * (Lg(2, g00) + Hg(2, g00)) + (Pv(2, wy, xm) + Pv(2, wy, xp)) +
                     (Pv(2, ym, wx) + Pv(2, yp, wx));
#define MXY(c) (Pv(c, yp, xp) - Pv(c, ym, xp) - Pv(c, yp, xm) + Pv(c, ym, xm))
#define MXZ(c) (Hg(c, gp0) - Lg(c, gp0) - Hg(c, gm0) + Lg(c, gm0))
#define MYZ(c) (Hg(c, g0p) - Lg(c, g0p) - Hg(c, g0m) + Lg(c, g0m))
        const T o0 = -(a0 + kq * (MXY(1) + MXZ(2)));
        const T o1 = -(a1 + kq * (MXY(0) + MYZ(2)));
        const T o2 = -(a2 + kq * (MXZ(0) + MYZ(1)));
        Pv(0, wy, wx) = (__ldg(v.B + g00) - o0) * f.dinv;
        Pv(1, wy, wx) = (__ldg(v.B + cs + g00) - o1) * f.dinv;
        Pv(2, wy, wx) = (__ldg(v.B + 2 * cs + g00) - o2) * f.dinv;
#undef Pv
#undef Lg
#undef Hg
#undef MXY
#undef MXZ
#undef MYZ
    }
};

// coarse levels: one constant 27-point stencil of 3x3 blocks (Eq. 36), in
// parity-class form
template <typename T>
struct CoarseOp {
    static constexpr bool kStageZ = false;
    Coarse<T> c;
    __device__ __forceinline__ void update(const View<T> &v, int wx, int wy) const {
        T o[3];
        auto u = [&](int b, int dx, int dy) -> T { return v.P[widx(b, wy + dy, wx + dx)]; };
        auto sd = [&](int b, int dx, int dy, T &S, T &D) {
            const int g = v.rowg[wy + dy] + v.colg[wx + dx];
            const T lo = __ldg(v.L + b * v.cs + g), hi = __ldg(v.H + b * v.cs + g);
            S = hi + lo;
            D = hi - lo;
        };
        coarse_plane_terms(c, u, o);
        coarse_z_terms(c, sd, o);
        const int g00 = v.rowg[wy] + v.colg[wx];
#pragma unroll
        for (int a = 0; a < 3; a++)
            v.P[widx(a, wy, wx)] = c.dinv[a] * (__ldg(v.B + a * v.cs + g00) - o[a]);
    }
};

// resident CTAs per SM the register budget is cut for: the 27-point operator
// needs more registers a thread than the 19-point one
template <class Op>
struct MinBlocks {
    static constexpr int value = 6;
};
template <>
struct MinBlocks<CoarseOp<float>> {
    static constexpr int value = 2;
};

// update the nodes of in-plane colour (pi, pj) inside window region
// [xa, xb) x [ya, yb)
template <typename T, class Op>
__device__ __forceinline__ void colour_pass(const View<T> &v, const Op &op, int pi, int pj,
                                            int xa, int xb, int ya, int yb) {
    const int ua = (xa - pi + 1) >> 1, ub = (xb - pi + 1) >> 1;
    const int wa = (ya - pj + 1) >> 1, wb = (yb - pj + 1) >> 1;
    const int nu = ub - ua, n = nu * (wb - wa);
    for (int t = threadIdx.x; t < n; t += NT) {
        const int wx = 2 * (ua + t % nu) + pi;
        const int wy = 2 * (wa + t / nu) + pj;
        op.update(v, wx, wy);
    }
}

// 2 x T in one aligned load (x0 - HX and nx are even)
template <typename T>
struct Pair;
template <>
struct Pair<float> {
    typedef float2 V;
};
template <>
struct Pair<double> {
    typedef double2 V;
};

// phase kernel: plane k = 2 * blockIdx.z + kbase, one TX x TY tile per CTA.
// F selects the in-plane colour order (F,F), (1-F,F), (F,1-F), (1-F,1-F) in
// (i, j) parity.  zsrc holds the z-neighbour planes (old values in the first
// phase, the first phase's output in the second).
template <typename T, class Op, int F>
__global__ void __launch_bounds__(NT, MinBlocks<Op>::value)
    k_gs_tiled(Dims d, Op op, const T *__restrict__ b, const T *__restrict__ vin,
               const T *__restrict__ zsrc, T *__restrict__ vout, int kbase, int split) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    constexpr bool SZ = Op::kStageZ;
    T *sP = reinterpret_cast<T *>(smem_raw);
    T *sL = sP + WIN, *sH = sP + 2 * WIN;  // used only when SZ
    int *colg = reinterpret_cast<int *>(sP + (SZ ? 3 : 1) * WIN), *rowg = colg + WX;
    typedef typename Pair<T>::V V2;
    const int nx = d.nx, ny = d.ny;
    const long ps = (long)nx * ny, cs = d.cs;
    const int x0 = blockIdx.x * TX, y0 = blockIdx.y * TY;
    const int k = 2 * blockIdx.z + kbase;
    const int hnx = nx >> 1;
    for (int e = threadIdx.x; e < WX + WY; e += NT) {
        if (e < WX) {
            const int gx = wrap_mod(x0 - HX + e, nx);
            colg[e] = split ? (gx & 1) * hnx + (gx >> 1) : gx;
        } else {
            rowg[e - WX] = wrap_mod(y0 - HY + (e - WX), ny) * nx;
        }
    }
    __syncthreads();
    // stage the plane's window (and, with SZ, its z-neighbours') as (even,
    // odd) column pairs: one aligned pair load, two conflict-free stores
    auto stage = [&](T *dst, const T *src) {
        if (!split) {
            for (int e = threadIdx.x; e < 3 * WY * WH; e += NT) {
                const int c = e / (WY * WH), r = e - c * (WY * WH);
                const int wy = r / WH, h = r - wy * WH;
                const V2 p2 =
                    __ldg(reinterpret_cast<const V2 *>(src + c * cs + rowg[wy] + colg[2 * h]));
                dst[widx(c, wy, 2 * h)] = p2.x;
                dst[widx(c, wy, 2 * h + 1)] = p2.y;
            }
        } else if ((hnx & 1) == 0) {
            // parity-split rows, nx a multiple of 4: the window's half-rows
            // are runs of aligned same-parity pairs (the periodic wrap falls
            // between pairs)
            for (int e = threadIdx.x; e < 3 * WY * WH; e += NT) {
                const int c = e / (WY * WH), r = e - c * (WY * WH);
                const int wy = r / WH, q = r - wy * WH;
                const int par = q / (WH / 2), h = 2 * (q - par * (WH / 2)), wx = 2 * h + par;
                const V2 p2 =
                    __ldg(reinterpret_cast<const V2 *>(src + c * cs + rowg[wy] + colg[wx]));
                dst[widx(c, wy, wx)] = p2.x;
                dst[widx(c, wy, wx + 2)] = p2.y;
            }
        } else {
            // parity-split rows, single values
            for (int e = threadIdx.x; e < 3 * WY * WX; e += NT) {
                const int c = e / (WY * WX), r = e - c * (WY * WX);
                const int wy = r / WX, q = r - wy * WX;
                const int par = q / WH, h = q - par * WH, wx = 2 * h + par;
                dst[widx(c, wy, wx)] = __ldg(src + c * cs + rowg[wy] + colg[wx]);
            }
        }
    };
    stage(sP, vin + (long)k * ps);
    if (SZ) {
        stage(sL, zsrc + (long)(k - 1) * ps);
        stage(sH, zsrc + (long)(k + 1) * ps);
    }
    __syncthreads();
    View<T> v;
    v.P = sP;
    v.L = zsrc + (long)(k - 1) * ps;
    v.H = zsrc + (long)(k + 1) * ps;
    v.B = b + (long)k * ps;
    v.cs = cs;
    v.rowg = rowg;
    v.colg = colg;
    v.Ls = sL;
    v.Hs = sH;
    // the 4 in-plane colours on shrinking regions (window coordinates; the
    // tile is [HX, HX+TX) x [HY, HY+TY))
    colour_pass<T, Op>(v, op, F, F, 1, WX - 1, 1, WY - 1);
    __syncthreads();
    colour_pass<T, Op>(v, op, 1 - F, F, 2, WX - 2, 1, WY - 1);
    __syncthreads();
    colour_pass<T, Op>(v, op, F, 1 - F, 3, WX - 3, 2, WY - 2);
    __syncthreads();
    colour_pass<T, Op>(v, op, 1 - F, 1 - F, 4, WX - 4, 2, WY - 2);
    __syncthreads();
    // store the tile (nodes inside the grid only)
    T *out = vout + (long)k * ps;
    if (!split) {
        for (int e = threadIdx.x; e < 3 * TY * (TX / 2); e += NT) {
            const int c = e / (TY * (TX / 2)), r = e - c * (TY * (TX / 2));
            const int ty = r / (TX / 2), h = r - ty * (TX / 2);
            const int gx = x0 + 2 * h, gy = y0 + ty;
            if (gx < nx && gy < ny) {
                V2 p2;
                p2.x = sP[widx(c, ty + HY, 2 * h + HX)];
                p2.y = sP[widx(c, ty + HY, 2 * h + HX + 1)];
                *reinterpret_cast<V2 *>(out + c * cs + (long)gy * nx + gx) = p2;
            }
        }
    } else if ((hnx & 1) == 0) {
        // pairs of same-parity nodes (x0/2 is even, so each pair is aligned)
        for (int e = threadIdx.x; e < 3 * TY * (TX / 2); e += NT) {
            const int c = e / (TY * (TX / 2)), r = e - c * (TY * (TX / 2));
            const int ty = r / (TX / 2), q = r - ty * (TX / 2);
            const int par = q / (TX / 4), h = 2 * (q - par * (TX / 4));
            const int gx = x0 + 2 * h + par, gy = y0 + ty;
            if (gx < nx && gy < ny) {
                V2 p2;
                p2.x = sP[widx(c, ty + HY, 2 * h + par + HX)];
                p2.y = sP[widx(c, ty + HY, 2 * h + par + 2 + HX)];
                *reinterpret_cast<V2 *>(out + c * cs + (long)gy * nx + par * hnx + (gx >> 1)) = p2;
            }
        }
    } else {
        for (int e = threadIdx.x; e < 3 * TY * TX; e += NT) {
            const int c = e / (TY * TX), r = e - c * (TY * TX);
            const int ty = r / TX, q = r - ty * TX;
            const int par = q / (TX / 2), h = q - par * (TX / 2);
            const int gx = x0 + 2 * h + par, gy = y0 + ty;
            if (gx < nx && gy < ny)
                out[c * cs + (long)gy * nx + par * hnx + (gx >> 1)] =
                    sP[widx(c, ty + HY, 2 * h + par + HX)];
        }
    }
}

template <typename T, class Op, int F>
cudaError_t launch_phase(const Dims &d, const Op &op, const T *b, const T *vin, const T *zsrc,
                         T *vout, int par, cudaStream_t s, int split) {
    // planes of parity par among the interior planes 1..nz-1
    const int kbase = par ? 1 : 2;
    const int nplanes = par ? d.nz / 2 : d.nz / 2 - 1;
    if (nplanes <= 0) return cudaSuccess;
    constexpr size_t smem = smem_bytes<T, Op::kStageZ>();
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(k_gs_tiled<T, Op, F>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
    }
    dim3 grid((d.nx + TX - 1) / TX, (d.ny + TY - 1) / TY, nplanes);
    k_gs_tiled<T, Op, F><<<grid, NT, smem, s>>>(d, op, b, vin, zsrc, vout, kbase, split);
    count_launch();
    return cudaGetLastError();
}

template <typename T, class Op>
cudaError_t sweep(const Dims &d, const Op &op, const T *b, const T *vin, T *vout,
                  bool descending, cudaStream_t s, int split) {
    cudaError_t e;
    if (!descending) {
        // colours 0-3 on the even planes, then 4-7 on the odd planes
        e = launch_phase<T, Op, 0>(d, op, b, vin, vin, vout, 0, s, split);
        if (e != cudaSuccess) return e;
        return launch_phase<T, Op, 0>(d, op, b, vin, vout, vout, 1, s, split);
    }
    // colours 7-4 on the odd planes, then 3-0 on the even planes
    e = launch_phase<T, Op, 1>(d, op, b, vin, vin, vout, 1, s, split);
    if (e != cudaSuccess) return e;
    return launch_phase<T, Op, 1>(d, op, b, vin, vout, vout, 0, s, split);
}


// ------------------------------------------------------------------------
// Whole-plane phase kernel for small coarse levels (planes of at most
// kPlaneMax nodes): one CTA per plane of the phase's parity holds the plane,
// its two z-neighbour planes and its right-hand side in shared memory
// ([component][ny][nx] each, 48 KB at 32 x 32), folds the z-neighbour terms
// into the right-hand side once, and runs the 4 in-plane colour passes on
// shared memory only, with periodic x, y indexing (no halo: the plane is
// whole).  The tile kernel, whose 72 x 20 window wraps several times around
// such small planes, spends ~15-17 us a launch on latency at these sizes;
// this kernel takes 10.7 us at 32 x 32 (one thread per node) and 6.4-6.7 us
// at 16 x 16 and 8 x 8 (measured on GB300).  At 64 x 64 it loses to the tile
// kernel (27.7 against 18 us: one CTA per plane leaves most SMs idle).
constexpr int kPlaneMax = 1024;
constexpr int kPlaneThreads = 1024;  // at most; one per node of the plane

template <int F>
__global__ void __launch_bounds__(kPlaneThreads)
    k_gs_plane(Dims d, Coarse<float> c, const float *__restrict__ b, const float *__restrict__ vin,
               const float *__restrict__ zsrc, float *__restrict__ vout, int kbase) {
    extern __shared__ __align__(16) float smp[];
    const int nx = d.nx, ny = d.ny, np = nx * ny;
    const long ps = (long)np, cs = d.cs;
    float *P = smp, *Lz = smp + 3 * np, *Hz = smp + 6 * np, *Rr = smp + 9 * np;
    const int k = 2 * blockIdx.x + kbase;
    for (int e = threadIdx.x; e < 3 * np; e += blockDim.x) {
        const int a = e / np, m = e - a * np;
        P[e] = vin[a * cs + k * ps + m];
        Lz[e] = zsrc[a * cs + (k - 1) * ps + m];
        Hz[e] = zsrc[a * cs + (k + 1) * ps + m];
        Rr[e] = b[a * cs + k * ps + m];
    }
    __syncthreads();
    // fold the z-neighbour blocks (dz = -1, +1) into the right-hand side
    for (int m = threadIdx.x; m < np; m += blockDim.x) {
        const int j = m / nx, i = m - j * nx;
        const int col[3] = {i ? i - 1 : nx - 1, i, i + 1 < nx ? i + 1 : 0};
        const int row[3] = {(j ? j - 1 : ny - 1) * nx, j * nx, (j + 1 < ny ? j + 1 : 0) * nx};
        auto sd = [&](int b, int dx, int dy, float &S, float &D) {
            const int q = b * np + row[dy + 1] + col[dx + 1];
            S = Hz[q] + Lz[q];
            D = Hz[q] - Lz[q];
        };
        float o[3] = {0.f, 0.f, 0.f};
        coarse_z_terms(c, sd, o);
        Rr[m] -= o[0];
        Rr[np + m] -= o[1];
        Rr[2 * np + m] -= o[2];
    }
    __syncthreads();
    // colours (F,F), (1-F,F), (F,1-F), (1-F,1-F) in (x, y) parity
    const int hx = nx >> 1, nh = np >> 2;
#pragma unroll 1
    for (int pass = 0; pass < 4; pass++) {
        const int pi = (pass & 1) ? 1 - F : F, pj = (pass & 2) ? 1 - F : F;
        for (int t = threadIdx.x; t < nh; t += blockDim.x) {
            const int jh = t / hx, i = 2 * (t - jh * hx) + pi, j = 2 * jh + pj;
            const int col[3] = {i ? i - 1 : nx - 1, i, i + 1 < nx ? i + 1 : 0};
            const int row[3] = {(j ? j - 1 : ny - 1) * nx, j * nx, (j + 1 < ny ? j + 1 : 0) * nx};
            auto u = [&](int b, int dx, int dy) -> float {
                return P[b * np + row[dy + 1] + col[dx + 1]];
            };
            float o[3];
            coarse_plane_terms(c, u, o);
            const int m = j * nx + i;
#pragma unroll
            for (int a = 0; a < 3; a++) P[a * np + m] = c.dinv[a] * (Rr[a * np + m] - o[a]);
        }
        __syncthreads();
    }
    for (int e = threadIdx.x; e < 3 * np; e += blockDim.x) {
        const int a = e / np, m = e - a * np;
        vout[a * cs + k * ps + m] = P[e];
    }
}

template <int F>
cudaError_t launch_plane(const Dims &d, const Coarse<float> &c, const float *b, const float *vin,
                         const float *zsrc, float *vout, int par, cudaStream_t s) {
    const int kbase = par ? 1 : 2;
    const int nplanes = par ? d.nz / 2 : d.nz / 2 - 1;
    if (nplanes <= 0) return cudaSuccess;
    const size_t smem = 12 * (size_t)d.nx * d.ny * sizeof(float);
    const int np = d.nx * d.ny;
    const int threads = np < kPlaneThreads ? ((np + 31) / 32) * 32 : kPlaneThreads;
    k_gs_plane<F><<<nplanes, threads, smem, s>>>(d, c, b, vin, zsrc, vout, kbase);
    count_launch();
    return cudaGetLastError();
}

}  // namespace

cudaError_t plane_init() {
    const int smem = (int)(12 * (size_t)kPlaneMax * sizeof(float));
    cudaError_t e = cudaFuncSetAttribute(k_gs_plane<0>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         smem);
    if (e != cudaSuccess) return e;
    return cudaFuncSetAttribute(k_gs_plane<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
}

// one 8-colour sweep vin -> vout (vout's wall planes must hold the walls)
cudaError_t gs_sweep_fine_tiled(const Dims &d, const Fine<float> &f, const float *b,
                                const float *vin, float *vout, bool descending, cudaStream_t s,
                                int split, const SweepSync *sync) {
    // whole rows per CTA where the rows are short enough (smoother_rows.cu)
    const cudaError_t e = gs_sweep_fine_rows(d, f, b, vin, vout, descending, s, split, sync);
    if (e != cudaErrorNotSupported) return e;
    FineOp<float> op{f};
    return sweep<float>(d, op, b, vin, vout, descending, s, split);
}

cudaError_t gs_sweep_coarse_tiled(const Dims &d, const Coarse<float> &c, const float *b,
                                  const float *vin, float *vout, bool descending, cudaStream_t s) {
    if ((long)d.nx * d.ny <= kPlaneMax) {
        // whole planes in shared memory
        cudaError_t e;
        if (!descending) {
            e = launch_plane<0>(d, c, b, vin, vin, vout, 0, s);
            if (e != cudaSuccess) return e;
            return launch_plane<0>(d, c, b, vin, vout, vout, 1, s);
        }
        e = launch_plane<1>(d, c, b, vin, vin, vout, 1, s);
        if (e != cudaSuccess) return e;
        return launch_plane<1>(d, c, b, vin, vout, vout, 0, s);
    }
    // whole-row strips where the rows fit (smoother_rows.cu)
    const cudaError_t e = gs_sweep_coarse_rows(d, c, b, vin, vout, descending, s);
    if (e != cudaErrorNotSupported) return e;
    CoarseOp<float> op{c};
    return sweep<float>(d, op, b, vin, vout, descending, s, 0);
}

}  // namespace qsmg

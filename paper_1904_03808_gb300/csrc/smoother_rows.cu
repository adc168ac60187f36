// smoother_rows.cu -- row-strip Gauss-Seidel sweep phases (FP32) for the
// finest level (structured 19-point operator of the scaled Eq. 30) and for
// coarse levels of rows >= 128 nodes (27-point block stencil, Eq. 36), and
// the finest-level residual.
//
// One 8-colour sweep runs as two phase launches, as in smoother_fast.cu:
// the planes of one k-parity (4 in-plane colours each, reading the old
// z-neighbour planes), then the planes of the other parity (reading the
// first phase's output).  Here a CTA owns whole rows of a plane, so the
// periodic x direction needs no halo.  Two kernels:
//   k_gs_rows_p  persistent, for rows of 64, 128, 192 or 256 nodes (a
//                multiple of 64, at least 9 rows): the rows of
//                each tile are copied into shared memory with cp.async while
//                the other CTAs on the SM compute; templated on the operator
//                (FineRowsOp, CoarseRowsOp) and, with RES, computing the
//                residual b - A x instead of a sweep phase (with RR as well,
//                restricting it in x and y on the fly instead of storing it);
//   k_gs_rows    one CTA per tile, operands loaded straight into registers,
//                for the other finest rows of up to 512 nodes.
// Both compute every node from the same neighbour values as the sequential
// colour order (tested against the eight colour launches).
#include <stdint.h>

#include "qsmg_impl.h"

namespace qsmg {
namespace {

__device__ __forceinline__ int wrap_mod(int a, int n) {
    a %= n;
    return a < 0 ? a + n : a;
}

// ------------------------------------------------------------------------
// Tile geometry shared by both kernels.  A CTA owns TY whole rows of one plane; thread t owns the node pair
// x = 2t ("E") and x = 2t+1 ("O") in every row of the strip's window and
// keeps their values in registers, so of a node's eight in-plane neighbours
// only the three on the far x side (the neighbouring thread's column) come
// through shared memory.  Whole rows need no x halo: the periodic x wrap is
// the neighbour index t-1 / t+1 modulo nx/2.
//
// Window rows jj = 0 .. TY+2 are y = y0 - 1 - F + jj.  With the colour order
// (F,F), (1-F,F), (F,1-F), (1-F,1-F) in (x, y) parity, the F-parity rows are
// the odd jj and the tile rows are jj = 1+F .. TY+F:
//   pass 1, 2: x-parity F, then 1-F, on the odd rows 1 .. TY+1 (reading the
//              old even rows around them);
//   pass 3, 4: x-parity F, then 1-F, on the even rows 2 .. TY.
// Every tile node then sees exactly the neighbour values of the sequential
// colour order; rows 0 and TY+2 are read only.
//
// The z-neighbour planes (old values in the first phase, the first phase's
// output in the second) do not change during a phase, so their contribution
// is folded into the right-hand side once per node before the passes:
//   r_c = b_c + z_c,
//   z_0 = (L0+H0) + kq (D2(x+1) - D2(x-1)),
//   z_1 = (L1+H1) + kq (D2(y+1) - D2(y-1)),
//   z_2 = lp (L2+H2) + kq ((D0(x+1) - D0(x-1)) + (D1(y+1) - D1(y-1))),
// with D = H - L, streamed row by row so each plane value is loaded once.
constexpr int kRowsMaxThreads = 256;  // rows up to 512 nodes

// numerators of the node of x-parity E at window row jj: the folded
// right-hand side r plus the in-plane neighbour terms, from the own column
// values P and the far-side neighbour column X[c * sc + row * sr + xn]
// (shared memory); the Gauss-Seidel update is numerator / d0, the residual
// numerator - d0 x
template <int E, int R>
__device__ __forceinline__ void rows_numer(const float (&P)[3][2][R], float r0, float r1,
                                           float r2, const float *X, int sc, int sr, int xn,
                                           int jj, const Fine<float> &f, float num[3]) {
    float m[3][3], p[3][3];  // [component][row jj-1, jj, jj+1] at x-1 and x+1
#pragma unroll
    for (int q = 0; q < 3; q++)
#pragma unroll
        for (int c = 0; c < 3; c++) {
            if (q != 1 && c == 2) continue;  // comp 2 enters only through row jj
            const float own = P[c][1 - E][jj - 1 + q];
            const float nb = X[c * sc + (jj - 1 + q) * sr + xn];
            if (E == 0) {
                p[c][q] = own;
                m[c][q] = nb;
            } else {
                m[c][q] = own;
                p[c][q] = nb;
            }
        }
    const float lp = f.lp, kq = f.kq;
    num[0] = r0 + lp * (m[0][1] + p[0][1]) + (P[0][E][jj - 1] + P[0][E][jj + 1]) +
             kq * (p[1][2] - p[1][0] - m[1][2] + m[1][0]);
    num[1] = r1 + lp * (P[1][E][jj - 1] + P[1][E][jj + 1]) + (m[1][1] + p[1][1]) +
             kq * (p[0][2] - p[0][0] - m[0][2] + m[0][0]);
    num[2] = r2 + (m[2][1] + p[2][1]) + (P[2][E][jj - 1] + P[2][E][jj + 1]);
}

// Gauss-Seidel update of the node of x-parity E at window row jj
template <int E, int R>
__device__ __forceinline__ void rows_update(float (&P)[3][2][R], float r0, float r1, float r2,
                                            const float *X, int sc, int sr, int xn, int jj,
                                            const Fine<float> &f) {
    float num[3];
    rows_numer<E, R>(P, r0, r1, r2, X, sc, sr, xn, jj, f, num);
#pragma unroll
    for (int c = 0; c < 3; c++) P[c][E][jj] = num[c] * f.dinv;
}

template <int TY, int F, bool SPLIT>
__global__ void __launch_bounds__(kRowsMaxThreads, 2)
    k_gs_rows(Dims d, Fine<float> f, const float *__restrict__ b, const float *__restrict__ vin,
              const float *__restrict__ zsrc, float *__restrict__ vout, int kbase) {
    constexpr int R = TY + 3;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int nt = blockDim.x;
    float *XE = reinterpret_cast<float *>(smem_raw);  // [3][R][nt] E values by column
    float *XO = XE + 3 * R * nt;                       // [3][R][nt] O values by column
    float *RS = XO + 3 * R * nt;                       // [3][2][R][nt] folded right-hand sides
    const int nx = d.nx, ny = d.ny, hn = nx >> 1;
    const long ps = (long)nx * ny, cs = d.cs;
    const int t = threadIdx.x;
    const bool act = t < hn;
    const int tc = act ? t : hn - 1;  // spare lanes mirror the last column, store nothing
    const int tm = tc == 0 ? hn - 1 : tc - 1, tp = tc + 1 == hn ? 0 : tc + 1;
    const int cE = SPLIT ? tc : 2 * tc, cO = SPLIT ? hn + tc : 2 * tc + 1;
    const int cOm = SPLIT ? hn + tm : 2 * tm + 1;  // x - 1 of the E node
    const int cEp = SPLIT ? tp : 2 * tp;           // x + 1 of the O node
    const int k = 2 * blockIdx.y + kbase;
    const int y0 = blockIdx.x * TY;
    const float lp = f.lp, kq = f.kq;

    // right-hand side with the z-neighbour terms folded in, for rows 1 .. R-2,
    // streamed row by row (row jj's plane values complete row jj-1)
    const float *Lz = zsrc + (long)(k - 1) * ps, *Hz = zsrc + (long)(k + 1) * ps;
    const float *Bk = b + (long)k * ps;
    float S1[3][2], D1[3][2];  // row jj-1: L+H and H-L of the own columns
    float D2y[2][2];           // row jj-2: H-L of components 1, 2
    float dm0 = 0.f, dm2 = 0.f, dp0 = 0.f, dp2 = 0.f;  // row jj-1: far-side H-L
#pragma unroll 2
    for (int jj = 0; jj < R; jj++) {
        const int o = wrap_mod(y0 - 1 - F + jj, ny) * nx;
        float S0[3][2], D0[3][2];
#pragma unroll
        for (int c = 0; c < 3; c++) {
            const float lE = __ldg(Lz + c * cs + o + cE), hE = __ldg(Hz + c * cs + o + cE);
            const float lO = __ldg(Lz + c * cs + o + cO), hO = __ldg(Hz + c * cs + o + cO);
            S0[c][0] = lE + hE;
            S0[c][1] = lO + hO;
            D0[c][0] = hE - lE;
            D0[c][1] = hO - lO;
        }
        const float nm0 = __ldg(Hz + o + cOm) - __ldg(Lz + o + cOm);
        const float nm2 = __ldg(Hz + 2 * cs + o + cOm) - __ldg(Lz + 2 * cs + o + cOm);
        const float np0 = __ldg(Hz + o + cEp) - __ldg(Lz + o + cEp);
        const float np2 = __ldg(Hz + 2 * cs + o + cEp) - __ldg(Lz + 2 * cs + o + cEp);
        if (jj >= 2) {
            const int ob = wrap_mod(y0 - 2 - F + jj, ny) * nx;
            const int w = jj - 1;
#define RSW(c, e) RS[(((c) * 2 + (e)) * R + w) * nt + t]
            // E node: x-1 is the neighbour's O column, x+1 the own O column
            RSW(0, 0) = __ldg(Bk + ob + cE) + (S1[0][0] + kq * (D1[2][1] - dm2));
            RSW(1, 0) = __ldg(Bk + cs + ob + cE) + (S1[1][0] + kq * (D0[2][0] - D2y[1][0]));
            RSW(2, 0) = __ldg(Bk + 2 * cs + ob + cE) +
                        (lp * S1[2][0] + kq * ((D1[0][1] - dm0) + (D0[1][0] - D2y[0][0])));
            // O node: x-1 is the own E column, x+1 the neighbour's E column
            RSW(0, 1) = __ldg(Bk + ob + cO) + (S1[0][1] + kq * (dp2 - D1[2][0]));
            RSW(1, 1) = __ldg(Bk + cs + ob + cO) + (S1[1][1] + kq * (D0[2][1] - D2y[1][1]));
            RSW(2, 1) = __ldg(Bk + 2 * cs + ob + cO) +
                        (lp * S1[2][1] + kq * ((dp0 - D1[0][0]) + (D0[1][1] - D2y[0][1])));
#undef RSW
        }
#pragma unroll
        for (int e = 0; e < 2; e++) {
            D2y[0][e] = D1[1][e];
            D2y[1][e] = D1[2][e];
#pragma unroll
            for (int c = 0; c < 3; c++) {
                S1[c][e] = S0[c][e];
                D1[c][e] = D0[c][e];
            }
        }
        dm0 = nm0;
        dm2 = nm2;
        dp0 = np0;
        dp2 = np2;
    }

    // own columns of this plane
    int roff[R];
#pragma unroll
    for (int jj = 0; jj < R; jj++) roff[jj] = wrap_mod(y0 - 1 - F + jj, ny) * nx;
    const float *Pk = vin + (long)k * ps;
    float P[3][2][R];
#pragma unroll
    for (int c = 0; c < 3; c++)
#pragma unroll
        for (int jj = 0; jj < R; jj++) {
            P[c][0][jj] = __ldg(Pk + c * cs + roff[jj] + cE);
            P[c][1][jj] = __ldg(Pk + c * cs + roff[jj] + cO);
        }

    // publish the own columns for the neighbours
#pragma unroll
    for (int c = 0; c < 3; c++)
#pragma unroll
        for (int jj = 0; jj < R; jj++) {
            XE[(c * R + jj) * nt + t] = P[c][0][jj];
            XO[(c * R + jj) * nt + t] = P[c][1][jj];
        }
    __syncthreads();
    // an E node's far side is column t-1's O, an O node's is column t+1's E
    constexpr int EF = F, EG = 1 - F;
    float *XF = EF == 0 ? XE : XO, *XG = EG == 0 ? XE : XO;
    const float *NF = EF == 0 ? XO : XE, *NG = EG == 0 ? XO : XE;
    const int tnF = EF == 0 ? tm : tp, tnG = EG == 0 ? tm : tp;
    // pass 1: x-parity F on the odd rows
#pragma unroll
    for (int jj = 1; jj < R - 1; jj += 2) {
        rows_update<EF, R>(P, RS[((0 * 2 + EF) * R + jj) * nt + t], RS[((1 * 2 + EF) * R + jj) * nt + t],
                               RS[((2 * 2 + EF) * R + jj) * nt + t], NF, R * nt, nt, tnF, jj, f);
#pragma unroll
        for (int c = 0; c < 3; c++) XF[(c * R + jj) * nt + t] = P[c][EF][jj];
    }
    __syncthreads();
    // pass 2: x-parity 1-F on the odd rows
#pragma unroll
    for (int jj = 1; jj < R - 1; jj += 2) {
        rows_update<EG, R>(P, RS[((0 * 2 + EG) * R + jj) * nt + t], RS[((1 * 2 + EG) * R + jj) * nt + t],
                               RS[((2 * 2 + EG) * R + jj) * nt + t], NG, R * nt, nt, tnG, jj, f);
#pragma unroll
        for (int c = 0; c < 3; c++) XG[(c * R + jj) * nt + t] = P[c][EG][jj];
    }
    __syncthreads();
    // pass 3: x-parity F on the even rows
#pragma unroll
    for (int jj = 2; jj < R - 2; jj += 2) {
        rows_update<EF, R>(P, RS[((0 * 2 + EF) * R + jj) * nt + t], RS[((1 * 2 + EF) * R + jj) * nt + t],
                               RS[((2 * 2 + EF) * R + jj) * nt + t], NF, R * nt, nt, tnF, jj, f);
#pragma unroll
        for (int c = 0; c < 3; c++) XF[(c * R + jj) * nt + t] = P[c][EF][jj];
    }
    __syncthreads();
    // pass 4: x-parity 1-F on the even rows
#pragma unroll
    for (int jj = 2; jj < R - 2; jj += 2) rows_update<EG, R>(P, RS[((0 * 2 + EG) * R + jj) * nt + t], RS[((1 * 2 + EG) * R + jj) * nt + t],
                               RS[((2 * 2 + EG) * R + jj) * nt + t], NG, R * nt, nt, tnG, jj, f);

    // store the tile rows
    if (!act) return;
    float *Ok = vout + (long)k * ps;
#pragma unroll
    for (int jj = 1 + F; jj < TY + 1 + F; jj++) {
        const int y = y0 - 1 - F + jj;
        if (y < ny) {
#pragma unroll
            for (int c = 0; c < 3; c++) {
                Ok[c * cs + roff[jj] + cE] = P[c][0][jj];
                Ok[c * cs + roff[jj] + cO] = P[c][1][jj];
            }
        }
    }
}

constexpr int kRowsTY = 6;  // tile rows: 128 registers without spills

// shared memory of one row-strip CTA: exchange columns (2 x 3 x R) and the
// folded right-hand sides (3 x 2 x R), nt columns each
inline size_t rows_smem(int nt) { return 12 * (size_t)(kRowsTY + 3) * nt * sizeof(float); }

template <int F, bool SPLIT>
cudaError_t launch_rows(const Dims &d, const Fine<float> &f, const float *b, const float *vin,
                        const float *zsrc, float *vout, int par, cudaStream_t s) {
    const int kbase = par ? 1 : 2;
    const int nplanes = par ? d.nz / 2 : d.nz / 2 - 1;
    if (nplanes <= 0) return cudaSuccess;
    const int nt = ((d.nx / 2 + 31) / 32) * 32;
    const size_t smem = rows_smem(nt);
    dim3 grid((d.ny + kRowsTY - 1) / kRowsTY, nplanes);
    k_gs_rows<kRowsTY, F, SPLIT><<<grid, nt, smem, s>>>(d, f, b, vin, zsrc, vout, kbase);
    count_launch();
    return cudaGetLastError();
}

template <int F>
cudaError_t rows_phase(const Dims &d, const Fine<float> &f, const float *b, const float *vin,
                       const float *zsrc, float *vout, int par, cudaStream_t s, int split) {
    return split ? launch_rows<F, true>(d, f, b, vin, zsrc, vout, par, s)
                 : launch_rows<F, false>(d, f, b, vin, zsrc, vout, par, s);
}


// ------------------------------------------------------------------------
// Persistent kernel.  Two CTAs per SM at nx = 256 (128 threads each; four at
// 128, eight at 64), each
// walking a contiguous run of the phase's tiles (strip, plane).  Tiles are
// ordered by blocks of kPersPB planes, then strip, then plane: consecutive
// tiles are mostly consecutive planes of one strip and share a z-neighbour
// plane (the upper plane of one tile is the lower plane of the next), and
// neighbouring strips reach the same plane within a few tiles, so the window
// rows they share are still in L2.  A tile's operands -- its plane's window
// rows, its right-hand-side rows and the window rows of its two z-neighbour
// planes -- are copied into shared memory with 16-byte cp.async copies
// issued when the previous tile is done (a z-plane slot already holding a
// needed plane is kept); the other CTA on the SM computes while they land.
// Shared rows are laid out [row][component][nx] in the arrays' own column
// order; the plane rows are updated in place and serve as the exchange
// buffer of the passes.  Copy lanes: thread t moves 16-byte chunk t % (nx/4)
// of the rows of parity t / (nx/4) (blockDim = nx/2 = 2 * nx/4).
// Measured on GB300 and dropped: one CTA per SM with double-buffered stages
// and four z-plane slots (24% slower); issuing the next tile's right-hand
// side and z-plane copies right after the first pass, when they are dead
// (6% slower, measured twice); right-hand-side rows loaded from global memory into
// registers instead of staged (freeing shared memory for taller tiles or a
// third CTA per SM: 10-17% slower); a cyclic plane-major tile order (27%
// fewer DRAM bytes, 18% slower: it loses the z-plane reuse); one thread per
// node component instead of per column pair (35% slower); natural instead of
// parity-split column order (8% slower); the prolongation x += T xc folded
// into the first post-sweep, each tile adding it to its copied input rows
// (the two launches took 323 + 158 us against 175 us for the plain sweep
// plus 146 us for the separate prolongation: every window row waits on its
// coarse loads from L2, with no registers or shared memory left to prefetch).
constexpr int kPersTY = 6;
constexpr int kPersR = kPersTY + 3;
constexpr int kPersMinBlocks = 2;  // resident CTAs per SM at nx = 256 (more for shorter rows)
constexpr int kPersMaxNx = 256;
constexpr int kPersPB = 16;  // planes per block of the tile order

__host__ __device__ constexpr long pers_floats(int nx) {
    return (long)(3 * kPersR + 3 * (kPersR - 2) + 2 * 3 * kPersR) * nx;
}

__device__ __forceinline__ void cp_async16(float *dst, const float *src) {
    const unsigned s = (unsigned)__cvta_generic_to_shared(dst);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() {
    asm volatile("cp.async.commit_group;\n" ::: "memory");
}
__device__ __forceinline__ void cp_async_wait_all() {
    asm volatile("cp.async.wait_group 0;\n" ::: "memory");
}

// Shared rows of a tile: [row][component][nx]; the own column pair of a
// thread is (xe, xo), the far-side neighbours xom (x - 1 of the E node) and
// xep (x + 1 of the O node).
struct RowCols {
    int nx, xe, xo, xom, xep;
    __device__ __forceinline__ int at(int row, int c, int x) const {
        return (row * 3 + c) * nx + x;
    }
};

// Finest level: the structured 19-point operator (scaled Eq. 30).
struct FineRowsOp {
    Fine<float> f;
    // right-hand side of window rows 1 .. R-2 with the z-neighbour terms
    // folded in (L, H: the lower and upper neighbour planes, B: b rows 1..R-2)
    template <int R>
    __device__ __forceinline__ void fold(float (&r)[3][2][R], const float *Ls, const float *Hs,
                                         const float *Bs, const RowCols &q) const {
        auto bv = [&](int jj, int c, int e) { return Bs[q.at(jj - 1, c, e ? q.xo : q.xe)]; };
        fold_with<R>(r, Ls, Hs, bv, q);
    }
    // the same with the right-hand side of window row jj, component c, node
    // e (0: E, 1: O) given by bv(jj, c, e)
    template <int R, class BV_>
    __device__ __forceinline__ void fold_with(float (&r)[3][2][R], const float *Ls,
                                              const float *Hs, const BV_ &bv,
                                              const RowCols &q) const {
        const float lp = f.lp, kq = f.kq;
        const int xe = q.xe, xo = q.xo, xom = q.xom, xep = q.xep;
#define DZ(row, c, x) (Hs[q.at(row, c, x)] - Ls[q.at(row, c, x)])
#define SZ(row, c, x) (Hs[q.at(row, c, x)] + Ls[q.at(row, c, x)])
#define BV(c, e) bv(jj, c, e)
#pragma unroll
        for (int jj = 1; jj < R - 1; jj++) {
            const float dOm0 = DZ(jj, 0, xom), dOm2 = DZ(jj, 2, xom);
            const float dEp0 = DZ(jj, 0, xep), dEp2 = DZ(jj, 2, xep);
            const float dE0 = DZ(jj, 0, xe), dE2 = DZ(jj, 2, xe);
            const float dO0 = DZ(jj, 0, xo), dO2 = DZ(jj, 2, xo);
            // E node: x-1 is the neighbour's O column, x+1 the own O column
            r[0][0][jj] = BV(0, 0) + (SZ(jj, 0, xe) + kq * (dO2 - dOm2));
            r[1][0][jj] =
                BV(1, 0) + (SZ(jj, 1, xe) + kq * (DZ(jj + 1, 2, xe) - DZ(jj - 1, 2, xe)));
            r[2][0][jj] = BV(2, 0) + (lp * SZ(jj, 2, xe) +
                                       kq * ((dO0 - dOm0) + (DZ(jj + 1, 1, xe) - DZ(jj - 1, 1, xe))));
            // O node: x-1 is the own E column, x+1 the neighbour's E column
            r[0][1][jj] = BV(0, 1) + (SZ(jj, 0, xo) + kq * (dEp2 - dE2));
            r[1][1][jj] =
                BV(1, 1) + (SZ(jj, 1, xo) + kq * (DZ(jj + 1, 2, xo) - DZ(jj - 1, 2, xo)));
            r[2][1][jj] = BV(2, 1) + (lp * SZ(jj, 2, xo) +
                                       kq * ((dEp0 - dE0) + (DZ(jj + 1, 1, xo) - DZ(jj - 1, 1, xo))));
        }
#undef DZ
#undef SZ
#undef BV
    }
    template <int E, int R>
    __device__ __forceinline__ void numer(const float (&P)[3][2][R], const float (&r)[3][2][R],
                                          const float *X, const RowCols &q, int jj,
                                          float num[3]) const {
        rows_numer<E, R>(P, r[0][E][jj], r[1][E][jj], r[2][E][jj], X, q.nx, 3 * q.nx,
                         E == 0 ? q.xom : q.xep, jj, f, num);
    }
    __device__ __forceinline__ void solve(const float num[3], float out[3]) const {
#pragma unroll
        for (int a = 0; a < 3; a++) out[a] = num[a] * f.dinv;
    }
    __device__ __forceinline__ void centre(const float x[3], float out[3]) const {
#pragma unroll
        for (int a = 0; a < 3; a++) out[a] = f.d0 * x[a];
    }
};

// Coarse levels: one constant 27-point stencil of 3x3 blocks (Galerkin
// product, Eq. 36), S[dd][a][b] with dd = 9 (dz+1) + 3 (dy+1) + (dx+1); the
// walls are zero planes, so the stencil needs no truncation here.  Coarse
// arrays are in natural column order, where a thread's E and O nodes are
// adjacent: every shared row is read as 8-byte (E, O) pairs -- the own pair
// and the pairs to the left (whose O is x - 1 of E) and right (whose E is
// x + 1 of O).
struct CoarseRowsOp {
    Coarse<float> c;
    __device__ __forceinline__ static float2 pair(const float *A, const RowCols &q, int row,
                                                  int comp, int x2) {
        return *reinterpret_cast<const float2 *>(&A[q.at(row, comp, x2)]);
    }
    template <int R>
    __device__ __forceinline__ void fold(float (&r)[3][2][R], const float *Ls, const float *Hs,
                                         const float *Bs, const RowCols &q) const {
        const int xl = q.xom - 1, xr = q.xep;  // first columns of the left / right pairs
#pragma unroll
        for (int jj = 1; jj < R - 1; jj++) {
            // z sums and differences at columns x_E - 1, x_E, x_O, x_O + 1
            float S[3][3][4], D[3][3][4];  // [component][dy + 1][column]
#pragma unroll
            for (int b = 0; b < 3; b++)
#pragma unroll
                for (int dy = -1; dy <= 1; dy++) {
                    const float2 ll = pair(Ls, q, jj + dy, b, xl), lo = pair(Ls, q, jj + dy, b, q.xe),
                                 lr = pair(Ls, q, jj + dy, b, xr);
                    const float2 hl = pair(Hs, q, jj + dy, b, xl), ho = pair(Hs, q, jj + dy, b, q.xe),
                                 hr = pair(Hs, q, jj + dy, b, xr);
                    const float L4[4] = {ll.y, lo.x, lo.y, lr.x}, H4[4] = {hl.y, ho.x, ho.y, hr.x};
#pragma unroll
                    for (int m = 0; m < 4; m++) {
                        S[b][dy + 1][m] = H4[m] + L4[m];
                        D[b][dy + 1][m] = H4[m] - L4[m];
                    }
                }
#pragma unroll
            for (int e = 0; e < 2; e++) {
                auto sd = [&](int b, int dx, int dy, float &s_, float &d_) {
                    s_ = S[b][dy + 1][e + dx + 1];
                    d_ = D[b][dy + 1][e + dx + 1];
                };
                float o[3] = {0.f, 0.f, 0.f};
                coarse_z_terms(c, sd, o);
#pragma unroll
                for (int a = 0; a < 3; a++) r[a][e][jj] = Bs[q.at(jj - 1, a, e ? q.xo : q.xe)] - o[a];
            }
        }
    }
    template <int E, int R>
    __device__ __forceinline__ void numer(const float (&P)[3][2][R], const float (&r)[3][2][R],
                                          const float *X, const RowCols &q, int jj,
                                          float num[3]) const {
        const int xfar = E == 0 ? q.xom - 1 : q.xep;  // the far-side neighbour's pair
        float far[3][3];                              // [component][dy + 1]
#pragma unroll
        for (int dy = -1; dy <= 1; dy++)
#pragma unroll
            for (int b = 0; b < 3; b++) {
                const float2 p2 = pair(X, q, jj + dy, b, xfar);
                far[b][dy + 1] = E == 0 ? p2.y : p2.x;
            }
        // x - 1 of E / x + 1 of O: the far-side column; otherwise the own E
        // (offset 0 of E, -1 of O) or the own O column
        auto u = [&](int b, int dx, int dy) -> float {
            if (E == 0 ? dx < 0 : dx > 0) return far[b][dy + 1];
            const int own = E == 0 ? (dx == 0 ? 0 : 1) : (dx == 0 ? 1 : 0);
            return P[b][own][jj + dy];
        };
        float o[3];
        coarse_plane_terms(c, u, o);
#pragma unroll
        for (int a = 0; a < 3; a++) num[a] = r[a][E][jj] - o[a];
    }
    __device__ __forceinline__ void solve(const float num[3], float out[3]) const {
#pragma unroll
        for (int a = 0; a < 3; a++) out[a] = c.dinv[a] * num[a];
    }
    __device__ __forceinline__ void centre(const float x[3], float out[3]) const {
#pragma unroll
        for (int a = 0; a < 3; a++) out[a] = c.cd[a][0] * x[a];
    }
};

// Gauss-Seidel update of the node of x-parity E at window row jj
template <int E, int R, class OP>
__device__ __forceinline__ void pers_update(const OP &op, float (&P)[3][2][R],
                                            const float (&r)[3][2][R], const float *X,
                                            const RowCols &q, int jj) {
    float num[3], out[3];
    op.template numer<E, R>(P, r, X, q, jj, num);
    op.solve(num, out);
#pragma unroll
    for (int c = 0; c < 3; c++) P[c][E][jj] = out[c];
}

// One sweep phase (or, with RES, the residual b - A x of every plane
// k = kbase, kbase + kstep, ...; then F = 0, vin = zsrc = x, vout = r).
// With RES and RR (F = 1) the residual is not stored: each tile applies the
// x and y parts of the restriction to it and vout receives, per fine plane,
// the coarse-grid partial sums [c][k][J][I] (c stride (nz+1) ny/2 nx/2) that
// k_restrict_z combines along z.
template <class OP, int F, bool SPLIT, bool RES, bool RR = false>
__global__ void __launch_bounds__(kPersMaxNx / 2, kPersMinBlocks)
    k_gs_rows_p(Dims d, OP op, const float *__restrict__ b, const float *__restrict__ vin,
                const float *__restrict__ zsrc, float *__restrict__ vout, int kbase, int kstep,
                int nplanes, int nstrips) {
    constexpr int TY = kPersTY, R = kPersR;
    extern __shared__ __align__(16) float sm[];
    const int nx = d.nx, ny = d.ny, hn = nx >> 1, cpr = nx >> 2;
    const long ps = (long)nx * ny, cs = d.cs;
    const int plane_f = 3 * R * nx, bst_f = 3 * (R - 2) * nx;
    float *const Ps = sm, *const Bs = sm + plane_f, *const Zs0 = Bs + bst_f;
    const int t = threadIdx.x;
    const int q4 = 4 * (t % cpr), g = t / cpr;
    const int tm = t == 0 ? hn - 1 : t - 1, tp = t + 1 == hn ? 0 : t + 1;
    RowCols q;
    q.nx = nx;
    q.xe = SPLIT ? t : 2 * t;
    q.xo = SPLIT ? hn + t : 2 * t + 1;
    q.xom = SPLIT ? hn + tm : 2 * tm + 1;
    q.xep = SPLIT ? tp : 2 * tp;
    const long ntiles = (long)nstrips * nplanes;
    const long n0 = blockIdx.x * ntiles / gridDim.x, n1 = (blockIdx.x + 1) * ntiles / gridDim.x;
    if (n0 >= n1) return;

    // window rows [jlo, jhi) of plane qq of src into dst (rows from jlo)
    auto copy_rows = [&](float *dst, const float *src, int qq, int y0, int jlo, int jhi) {
        const float *base = src + (long)qq * ps + q4;
        for (int jj = jlo + g; jj < jhi; jj += 2) {
            int y = y0 - 1 - F + jj;  // ny >= R: at most one wrap
            y = y < 0 ? y + ny : (y >= ny ? y - ny : y);
            const float *srow = base + (long)y * nx;
            float *drow = dst + (jj - jlo) * 3 * nx + q4;
            cp_async16(drow, srow);
            cp_async16(drow + nx, srow + cs);
            cp_async16(drow + 2 * nx, srow + 2 * cs);
        }
    };
    // tile n -> strip s, plane k
    auto tile_of = [&](long n, int &s, int &k) {
        const int blk = (int)(n / ((long)nstrips * kPersPB));
        const int pb = nplanes - blk * kPersPB < kPersPB ? nplanes - blk * kPersPB : kPersPB;
        const int rem = (int)(n - (long)blk * nstrips * kPersPB);
        s = rem / pb;
        k = kstep * (blk * kPersPB + rem - s * pb) + kbase;
    };
    // z-plane slots 0, 1 (tag: strip * (nz + 1) + plane; uniform over the CTA)
    int tag0 = -1, tag1 = -1;
    // right-hand-side rows and z-neighbour planes of tile n (a slot holding a
    // needed plane is kept, the other one refilled)
    auto issue_bz = [&](long n, int &sL, int &sH) {
        int s, k;
        tile_of(n, s, k);
        const int y0 = s * TY;
        copy_rows(Bs, b, k, y0, 1, R - 1);
        const int keyL = s * (d.nz + 1) + k - 1, keyH = keyL + 2;
        sL = tag0 == keyL ? 0 : (tag1 == keyL ? 1 : -1);
        sH = tag0 == keyH ? 0 : (tag1 == keyH ? 1 : -1);
        if (sL < 0) {
            sL = sH == 0 ? 1 : 0;
            if (sL == 0)
                tag0 = keyL;
            else
                tag1 = keyL;
            copy_rows(Zs0 + sL * plane_f, zsrc, k - 1, y0, 0, R);
        }
        if (sH < 0) {
            sH = 1 - sL;
            if (sH == 0)
                tag0 = keyH;
            else
                tag1 = keyH;
            copy_rows(Zs0 + sH * plane_f, zsrc, k + 1, y0, 0, R);
        }
        cp_async_commit();
    };
    // plane rows of tile n
    auto issue_p = [&](long n) {
        int s, k;
        tile_of(n, s, k);
        copy_rows(Ps, vin, k, s * TY, 0, R);
        cp_async_commit();
    };

    int sL, sH;
    issue_bz(n0, sL, sH);
    issue_p(n0);
    for (long n = n0; n < n1; n++) {
        cp_async_wait_all();
        __syncthreads();
        int s, k;
        tile_of(n, s, k);
        const int y0 = s * TY;
        // right-hand side with the z-neighbour terms folded in
        float r[3][2][R];
        op.template fold<R>(r, Zs0 + sL * plane_f, Zs0 + sH * plane_f, Bs, q);
        float P[3][2][R];
#pragma unroll
        for (int c = 0; c < 3; c++)
#pragma unroll
            for (int jj = 0; jj < R; jj++) {
                if (SPLIT) {
                    P[c][0][jj] = Ps[q.at(jj, c, q.xe)];
                    P[c][1][jj] = Ps[q.at(jj, c, q.xo)];
                } else {  // adjacent: one 8-byte load
                    const float2 v = *reinterpret_cast<const float2 *>(&Ps[q.at(jj, c, q.xe)]);
                    P[c][0][jj] = v.x;
                    P[c][1][jj] = v.y;
                }
            }
        if (RES) {
            // residual of the tile rows 1 .. TY: numerator - centre block x
            // (with RR rows 1 .. TY + 1, i.e. y0 - 1 .. y0 + TY - 1: the fine
            // rows of the strip's coarse rows)
            constexpr int NR = RR ? TY + 2 : TY + 1;
            float res[3][2][NR];
#pragma unroll
            for (int jj = 1; jj < NR; jj++) {
                float num[3], x[3], cx[3];
                op.template numer<0, R>(P, r, Ps, q, jj, num);
#pragma unroll
                for (int c = 0; c < 3; c++) x[c] = P[c][0][jj];
                op.centre(x, cx);
#pragma unroll
                for (int c = 0; c < 3; c++) res[c][0][jj] = num[c] - cx[c];
                op.template numer<1, R>(P, r, Ps, q, jj, num);
#pragma unroll
                for (int c = 0; c < 3; c++) x[c] = P[c][1][jj];
                op.centre(x, cx);
#pragma unroll
                for (int c = 0; c < 3; c++) res[c][1][jj] = num[c] - cx[c];
            }
            if (RR) {
                // full weighting R = T^T (weight 1 at offset 0, 1/2 at +-1 per
                // axis), x and y parts: coarse column I = t takes fine
                // x = 2t - 1 (the O node of thread t - 1), 2t, 2t + 1; coarse
                // row J = y0/2 + jc takes fine rows 2J - 1 .. 2J + 1, window
                // rows 2 jc + 1 .. 2 jc + 3.  The O residuals go through the
                // (now dead) plane rows in shared memory.
                __syncthreads();
                float *Xo = Ps;
#pragma unroll
                for (int c = 0; c < 3; c++)
#pragma unroll
                    for (int jj = 1; jj < NR; jj++) Xo[(c * NR + jj) * hn + t] = res[c][1][jj];
                __syncthreads();
                const int hny = ny >> 1;
                const long pcs = (long)(d.nz + 1) * hny * hn;
#pragma unroll
                for (int c = 0; c < 3; c++) {
                    float rx[NR];
#pragma unroll
                    for (int jj = 1; jj < NR; jj++)
                        rx[jj] = (0.5f * Xo[(c * NR + jj) * hn + tm] + res[c][0][jj]) +
                                 0.5f * res[c][1][jj];
#pragma unroll
                    for (int jc = 0; jc < TY / 2; jc++) {
                        const int J = (y0 >> 1) + jc;
                        if (J < hny)
                            vout[c * pcs + ((long)k * hny + J) * hn + t] =
                                (0.5f * rx[2 * jc + 1] + rx[2 * jc + 2]) + 0.5f * rx[2 * jc + 3];
                    }
                }
            } else {
#pragma unroll
                for (int c = 0; c < 3; c++)
#pragma unroll
                    for (int jj = 1; jj < TY + 1; jj++) {
                        P[c][0][jj] = res[c][0][jj];
                        P[c][1][jj] = res[c][1][jj];
                    }
            }
        } else {
            constexpr int EF = F, EG = 1 - F;
            const int xF = EF == 0 ? q.xe : q.xo, xG = EG == 0 ? q.xe : q.xo;
            // pass 1: x-parity F on the odd rows
#pragma unroll
            for (int jj = 1; jj < R - 1; jj += 2) {
                pers_update<EF, R>(op, P, r, Ps, q, jj);
#pragma unroll
                for (int c = 0; c < 3; c++) Ps[q.at(jj, c, xF)] = P[c][EF][jj];
            }
            __syncthreads();
            // pass 2: x-parity 1-F on the odd rows
#pragma unroll
            for (int jj = 1; jj < R - 1; jj += 2) {
                pers_update<EG, R>(op, P, r, Ps, q, jj);
#pragma unroll
                for (int c = 0; c < 3; c++) Ps[q.at(jj, c, xG)] = P[c][EG][jj];
            }
            __syncthreads();
            // pass 3: x-parity F on the even rows
#pragma unroll
            for (int jj = 2; jj < R - 2; jj += 2) {
                pers_update<EF, R>(op, P, r, Ps, q, jj);
#pragma unroll
                for (int c = 0; c < 3; c++) Ps[q.at(jj, c, xF)] = P[c][EF][jj];
            }
            __syncthreads();
            // pass 4: x-parity 1-F on the even rows
#pragma unroll
            for (int jj = 2; jj < R - 2; jj += 2) pers_update<EG, R>(op, P, r, Ps, q, jj);
        }
        // store the tile rows
        float *Ok = vout + (long)k * ps;
#pragma unroll
        for (int jj = 1 + F; jj < TY + 1 + F; jj++) {
            const int y = y0 - 1 - F + jj;
            if (!RR && y < ny) {
#pragma unroll
                for (int c = 0; c < 3; c++) {
                    Ok[c * cs + (long)y * nx + q.xe] = P[c][0][jj];
                    Ok[c * cs + (long)y * nx + q.xo] = P[c][1][jj];
                }
            }
        }
        if (n + 1 < n1) {
            // refill once every thread is done with this tile
            __syncthreads();
            issue_bz(n + 1, sL, sH);
            issue_p(n + 1);
        }
    }
}

int g_sms[64];  // SM count per device, set by smoother_init

// resident CTAs of the persistent kernel per SM: shared memory and registers
// scale with the row length (two CTAs at nx = 256, four at 128, eight at 64)
inline long pers_slots(int nx, int sms) {
    return (long)sms * kPersMinBlocks * (kPersMaxNx / nx);
}

template <class OP, int F, bool SPLIT, bool RES, bool RR = false>
cudaError_t launch_rows_p(const Dims &d, const OP &op, const float *b, const float *vin,
                          const float *zsrc, float *vout, int kbase, int kstep, int nplanes,
                          cudaStream_t s, int sms) {
    if (nplanes <= 0) return cudaSuccess;
    const int nstrips = (d.ny + kPersTY - 1) / kPersTY;
    const long ntiles = (long)nstrips * nplanes;
    const long slots = pers_slots(d.nx, sms);
    const int grid = (int)(ntiles < slots ? ntiles : slots);
    k_gs_rows_p<OP, F, SPLIT, RES, RR><<<grid, d.nx / 2, pers_floats(d.nx) * sizeof(float), s>>>(
        d, op, b, vin, zsrc, vout, kbase, kstep, nplanes, nstrips);
    count_launch();
    return cudaGetLastError();
}

// one sweep: the planes of one parity, then the other (ascending: even
// planes 2 .. nz-2 with colours 0-3, then odd planes 1 .. nz-1 with 4-7;
// descending: odd planes with 7-4, then even planes with 3-0)
template <class OP, bool SPLIT>
cudaError_t rows_p_sweep(const Dims &d, const OP &op, const float *b, const float *vin,
                         float *vout, bool descending, cudaStream_t s, int sms) {
    const int ne = d.nz / 2 - 1, no = d.nz / 2;
    cudaError_t e;
    if (!descending) {
        e = launch_rows_p<OP, 0, SPLIT, false>(d, op, b, vin, vin, vout, 2, 2, ne, s, sms);
        if (e != cudaSuccess) return e;
        return launch_rows_p<OP, 0, SPLIT, false>(d, op, b, vin, vout, vout, 1, 2, no, s, sms);
    }
    e = launch_rows_p<OP, 1, SPLIT, false>(d, op, b, vin, vin, vout, 1, 2, no, s, sms);
    if (e != cudaSuccess) return e;
    return launch_rows_p<OP, 1, SPLIT, false>(d, op, b, vin, vout, vout, 2, 2, ne, s, sms);
}

// ------------------------------------------------------------------------
// Fused sweep: both phases of an 8-colour sweep in one launch, so that each
// value of v comes from DRAM once per sweep instead of once per phase.  The
// planes of the first phase ("A": the even planes, colours 0-3, in an
// ascending sweep; the odd ones, colours 7-4, in a descending sweep) depend
// only on the sweep's input; a plane of the second phase ("B") needs the new
// values of the A planes just below and above it.  Number the A planes by
// step m = 1, 2, ...: kA(m) = kA0 + 2 (m - 1), and let B plane kB(m) =
// kA(m) - 1 go with it; B(m) needs A(m - 1) and A(m).
//
// Each CTA owns one row strip and runs over short chunks of steps along z:
// in chunk [m0, m1) it updates the strip's tiles of A planes m0 .. m1-1,
// then those of B planes m0 .. m1-1.  A B tile reads its own old plane
// (which the A tiles of the chunk just read as a z-neighbour) and the new A
// planes around it (which the chunk, its neighbouring strips' chunks and the
// chunk below just wrote), so both mostly come from L2; only b and the old A
// planes come from DRAM.  The tile loop is the persistent kernel's: each
// tile's operands are copied into shared memory while the previous tile is
// computed, with the z-plane slots reused between consecutive tiles.  Before
// copying a new A plane's window rows, a CTA waits for the ready flags of the
// strips that own them (published after each A tile's store by a barrier
// and a release store; read with a relaxed load a tile ahead, then again
// with an acquire
// load once seen set).  The steps are cut into fused_rounds bands of K
// chunks each; in round r the K CTAs of a strip take the K chunks of band r,
// the l-th CTA chunk (l + r) mod K (rotated so that the CTAs' loads match),
// so a B tile waits only on A tiles of the same or an earlier round,
// whose CTAs are running or done: the cooperative launch keeps every CTA
// resident, and no A tile waits on anything.  Every wait is bounded
// and sets the error word when it gives up (the sweep then carries on with
// what it read, and the host reports the error).
//
// Measured on GB300 against the two-launch sweep (k_gs_rows_p): 33 against
// 49 B of DRAM traffic a node and an L2 hit rate of 63 against 12%, but
// 0.199 against 0.178 ms a 256^3 sweep (0.108 against 0.101 at
// 256 x 256 x 128).  Both kernels are latency-bound at 8 warps an SM (no
// unit above 53% of its peak), so the DRAM they save buys no time, and the
// flag reads, the extra barrier of a B tile and the shorter runs of z-plane
// reuse cost about 10%.  Selected by MG_FLAG_FUSED_SWEEP; the two-launch
// sweep stays the default.

constexpr long kSpinMax = 1L << 22;  // flag polls before a wait gives up (about 2 s)
// chunks per CTA: enough that the A planes a chunk writes are still in L2
// when its B tiles read them (about 2-3 steps a chunk)
__host__ __device__ constexpr int fused_rounds(int nsteps) { return nsteps >= 128 ? 8 : 4; }

__device__ __forceinline__ int ld_acquire(const int *p) {
    int v;
    asm volatile("ld.acquire.gpu.global.s32 %0, [%1];\n" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ int ld_relaxed(const int *p) {
    int v;
    asm volatile("ld.relaxed.gpu.global.s32 %0, [%1];\n" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void st_release(int *p, int v) {
    asm volatile("st.release.gpu.global.s32 [%0], %1;\n" ::"l"(p), "r"(v) : "memory");
}
// wait until *f >= want, polling at most kSpinMax times; on giving up (or if
// another wait already gave up) set / leave the error word and return
__device__ __forceinline__ void wait_flag(const int *f, int want, int *err) {
    for (long it = 0; it < kSpinMax; it++) {
        if (ld_acquire(f) >= want) return;
        if (*(volatile int *)err) return;
        __nanosleep(64);
    }
    atomicOr(err, 1);
}

template <int F, bool SPLIT>
__global__ void __launch_bounds__(kPersMaxNx / 2, kPersMinBlocks)
    k_gs_rows_f(Dims d, FineRowsOp op, const float *__restrict__ b, const float *__restrict__ vin,
                float *__restrict__ vout, int kA0, int nsteps, int nstrips, int K, SweepSync sy) {
    constexpr int TY = kPersTY, R = kPersR;
    extern __shared__ __align__(16) float sm[];
    __shared__ int s_epoch;
    const int nx = d.nx, ny = d.ny, nz = d.nz, hn = nx >> 1, cpr = nx >> 2;
    const long ps = (long)nx * ny, cs = d.cs;
    const int plane_f = 3 * R * nx, bst_f = 3 * (R - 2) * nx;
    float *const Ps = sm, *const Bs = sm + plane_f, *const Zs0 = Bs + bst_f;
    const int t = threadIdx.x;
    const int q4 = 4 * (t % cpr), g = t / cpr;
    const int tm = t == 0 ? hn - 1 : t - 1, tp = t + 1 == hn ? 0 : t + 1;
    RowCols q;
    q.nx = nx;
    q.xe = SPLIT ? t : 2 * t;
    q.xo = SPLIT ? hn + t : 2 * t + 1;
    q.xom = SPLIT ? hn + tm : 2 * tm + 1;
    q.xep = SPLIT ? tp : 2 * tp;
    const int s = blockIdx.x % nstrips, lane = blockIdx.x / nstrips;
    const int y0 = s * TY;
    const int NR = fused_rounds(nsteps);
    if (t == 0) s_epoch = *(volatile int *)sy.epoch;
    __syncthreads();
    const int want = s_epoch + 1;

    // the CTA's tiles in order: round r (chunk lane + K r), phase ph (0: A,
    // 1: B), i-th tile of the run; step m, plane k.  An A run starts with the
    // chunk's last step, which the chunk above needs first, then goes up from
    // m0; a B run goes up from m0.  Valid A tiles have kA <= nz - 1, valid B
    // tiles kB >= 1
    struct Tile {
        int r, ph, i, m, m0, m1, k;
    };
    // round r covers band r of the steps, split into K chunks; the CTA of
    // lane l takes chunk (l + r) mod K, so that every CTA's chunks add up to
    // the same length within a step, and the chunk below a chunk (the
    // previous one of the band, or the last one of the band below) is taken
    // in the same round or the round before
    auto chunk_of = [&](Tile &U) {
        const int b0 = 1 + (int)((long)U.r * nsteps / NR);
        const int bl = 1 + (int)((long)(U.r + 1) * nsteps / NR) - b0;
        const int j = (lane + U.r) % K;
        U.m0 = b0 + j * bl / K;
        U.m1 = b0 + (j + 1) * bl / K;
    };
    auto step_of = [&](const Tile &U) {
        return U.ph == 1 ? U.m0 + U.i : (U.i == 0 ? U.m1 - 1 : U.m0 + U.i - 1);
    };
    auto plane_of = [&](const Tile &U) { return kA0 + 2 * (U.m - 1) - U.ph; };
    // the next valid tile after U (U.r == NR: none)
    auto advance = [&](Tile &U) {
        for (;;) {
            if (++U.i >= U.m1 - U.m0) {
                if (U.ph == 0) {
                    U.ph = 1;
                } else {
                    U.ph = 0;
                    if (++U.r >= NR) return;
                    chunk_of(U);
                }
                U.i = 0;
            }
            U.m = step_of(U);
            U.k = plane_of(U);
            if (U.k >= 1 && U.k <= nz - 1) return;
        }
    };
    auto wrow = [&](int jj) {
        const int y = y0 - 1 - F + jj;
        return y < 0 ? y + ny : (y >= ny ? y - ny : y);
    };
    // window rows [jlo, jhi) of plane qq of src into dst (rows from jlo)
    auto copy_rows = [&](float *dst, const float *src, int qq, int jlo, int jhi) {
        const float *base = src + (long)qq * ps + q4;
        for (int jj = jlo + g; jj < jhi; jj += 2) {
            const float *srow = base + (long)wrow(jj) * nx;
            float *drow = dst + (jj - jlo) * 3 * nx + q4;
            cp_async16(drow, srow);
            cp_async16(drow + nx, srow + cs);
            cp_async16(drow + 2 * nx, srow + 2 * cs);
        }
    };
    // z-plane slots 0, 1 (tag: plane; within one sweep a plane number is
    // always read from the same array: A tiles read old B planes from vin,
    // B tiles new A planes (or the walls) from vout)
    int tag0 = -1, tag1 = -1;
    // the strips owning the window rows (at most 3; fixed for the CTA)
    int own[3] = {-1, -1, -1}, nown = 0;
    for (int jj = 0; jj < R; jj++) {
        const int o = wrow(jj) / TY;
        if (nown < 3 && (nown == 0 || (own[nown - 1] != o && own[0] != o))) own[nown++] = o;
    }
    // the ready flag for thread idx before a tile's new z-neighbour planes
    // are copied: for a B tile, those (strip o, step mm) of the owners of
    // each A plane p = kA(mm) that is not already in a slot (walls need
    // none); at most 2 planes x 3 owners, one per thread idx < count
    auto flag_of = [&](const Tile &U, int idx) -> const int * {
        if (U.r >= NR || U.ph != 1 || idx >= 2 * nown) return nullptr;
        const int side = idx / nown, o = own[idx - side * nown];
        const int p = side ? U.k + 1 : U.k - 1, mm = side ? U.m : U.m - 1;
        if (p <= 0 || p >= nz || tag0 == p || tag1 == p) return nullptr;
        return sy.aflag + (long)o * (nsteps + 1) + mm;
    };
    // whether a B tile needs any flag (the same answer in every thread)
    auto needs_flags = [&](const Tile &U) {
        if (U.ph != 1) return false;
        const int pl = U.k - 1, ph_ = U.k + 1;
        return (pl > 0 && tag0 != pl && tag1 != pl) || (ph_ < nz && tag0 != ph_ && tag1 != ph_);
    };
    // copies of tile U's operands; fp / fv: this thread's flag for U and the
    // value it read from it earlier (checked, and waited for if not yet set,
    // before the z-plane copies that depend on it)
    auto issue_bz = [&](const Tile &U, int &sL, int &sH, const int *fp, int fv) {
        const int k = U.k;
        const float *zsrc = U.ph == 0 ? vin : vout;
        copy_rows(Bs, b, k, 1, R - 1);
        copy_rows(Ps, vin, k, 0, R);
        if (needs_flags(U)) {
            // fv was read a tile ahead without ordering (wait only if it was
            // not yet set); the acquire load orders this thread's (and,
            // through the barrier, the CTA's) later reads after the
            // producer's stores without waiting for this thread's own
            // copies in flight
            if (fp) {
                if (fv < want) wait_flag(fp, want, sy.err);
                (void)ld_acquire(fp);
            }
            __syncthreads();
        }
        sL = tag0 == k - 1 ? 0 : (tag1 == k - 1 ? 1 : -1);
        sH = tag0 == k + 1 ? 0 : (tag1 == k + 1 ? 1 : -1);
        if (sL < 0) {
            sL = sH == 0 ? 1 : 0;
            if (sL == 0)
                tag0 = k - 1;
            else
                tag1 = k - 1;
            copy_rows(Zs0 + sL * plane_f, zsrc, k - 1, 0, R);
        }
        if (sH < 0) {
            sH = 1 - sL;
            if (sH == 0)
                tag0 = k + 1;
            else
                tag1 = k + 1;
            copy_rows(Zs0 + sH * plane_f, zsrc, k + 1, 0, R);
        }
        cp_async_commit();
    };

    Tile T;
    T.r = 0;
    T.ph = 0;
    T.i = -1;
    chunk_of(T);
    advance(T);
    int sL = 0, sH = 1;
    if (T.r < NR) {
        const int *fp = flag_of(T, t);
        issue_bz(T, sL, sH, fp, fp ? ld_relaxed(fp) : want);
    }
    while (T.r < NR) {
        cp_async_wait_all();
        __syncthreads();
        // the next tile, and a first read of its flags (one per thread), in
        // flight while this tile is computed
        Tile Tn = T;
        advance(Tn);
        const int *fp = flag_of(Tn, t);
        const int fv = fp ? ld_relaxed(fp) : want;
        float r[3][2][R];
        op.template fold<R>(r, Zs0 + sL * plane_f, Zs0 + sH * plane_f, Bs, q);
        float P[3][2][R];
#pragma unroll
        for (int c = 0; c < 3; c++)
#pragma unroll
            for (int jj = 0; jj < R; jj++) {
                if (SPLIT) {
                    P[c][0][jj] = Ps[q.at(jj, c, q.xe)];
                    P[c][1][jj] = Ps[q.at(jj, c, q.xo)];
                } else {
                    const float2 v = *reinterpret_cast<const float2 *>(&Ps[q.at(jj, c, q.xe)]);
                    P[c][0][jj] = v.x;
                    P[c][1][jj] = v.y;
                }
            }
        constexpr int EF = F, EG = 1 - F;
        const int xF = EF == 0 ? q.xe : q.xo, xG = EG == 0 ? q.xe : q.xo;
#pragma unroll
        for (int jj = 1; jj < R - 1; jj += 2) {
            pers_update<EF, R>(op, P, r, Ps, q, jj);
#pragma unroll
            for (int c = 0; c < 3; c++) Ps[q.at(jj, c, xF)] = P[c][EF][jj];
        }
        __syncthreads();
#pragma unroll
        for (int jj = 1; jj < R - 1; jj += 2) {
            pers_update<EG, R>(op, P, r, Ps, q, jj);
#pragma unroll
            for (int c = 0; c < 3; c++) Ps[q.at(jj, c, xG)] = P[c][EG][jj];
        }
        __syncthreads();
#pragma unroll
        for (int jj = 2; jj < R - 2; jj += 2) {
            pers_update<EF, R>(op, P, r, Ps, q, jj);
#pragma unroll
            for (int c = 0; c < 3; c++) Ps[q.at(jj, c, xF)] = P[c][EF][jj];
        }
        __syncthreads();
#pragma unroll
        for (int jj = 2; jj < R - 2; jj += 2) pers_update<EG, R>(op, P, r, Ps, q, jj);
        float *Ok = vout + (long)T.k * ps;
#pragma unroll
        for (int jj = 1 + F; jj < TY + 1 + F; jj++) {
            const int y = y0 - 1 - F + jj;
            if (y < ny) {
#pragma unroll
                for (int c = 0; c < 3; c++) {
                    Ok[c * cs + (long)y * nx + q.xe] = P[c][0][jj];
                    Ok[c * cs + (long)y * nx + q.xo] = P[c][1][jj];
                }
            }
        }
        // every thread is done with this tile: publish an A tile, refill
        __syncthreads();
        if (T.ph == 0 && t == 0) st_release(sy.aflag + (long)s * (nsteps + 1) + T.m, want);
        T = Tn;
        if (T.r < NR) issue_bz(T, sL, sH, fp, fv);
    }
    cp_async_wait_all();
    __syncthreads();
    // the last CTA to finish advances the launch count
    if (t == 0) {
        __threadfence();
        if (atomicAdd(sy.done, 1) == (int)gridDim.x - 1) {
            atomicExch(sy.done, 0);
            __threadfence();
            atomicExch(sy.epoch, want);
        }
    }
}

// co-resident CTAs of the fused kernel per device and row length (64, 128,
// 192, 256 nodes; set by smoother_init)
int g_fused_slots[64][kPersMaxNx / 64];

inline int fused_nstrips(const Dims &d) { return (d.ny + kPersTY - 1) / kPersTY; }

// CTAs per strip: as many as fit beside the other strips' with all CTAs
// co-resident, so that every chunk has at least one step
inline int fused_k(const Dims &d, int slots) {
    const int nsteps = d.nz / 2, ns = fused_nstrips(d);
    int k = slots / ns;
    const int kmax = nsteps / fused_rounds(nsteps);
    return k < 1 || kmax < 1 ? 0 : (k > kmax ? kmax : k);
}

template <int F, bool SPLIT>
cudaError_t launch_fused(const Dims &d, const FineRowsOp &op, const float *b, const float *vin,
                         float *vout, int kA0, int K, const SweepSync &sy, cudaStream_t s) {
    const int nsteps = d.nz / 2, ns = fused_nstrips(d);
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(ns * K);
    cfg.blockDim = dim3(d.nx / 2);
    cfg.dynamicSmemBytes = pers_floats(d.nx) * sizeof(float);
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    const cudaError_t e = cudaLaunchKernelEx(&cfg, k_gs_rows_f<F, SPLIT>, d, op, b, vin, vout, kA0,
                                             nsteps, ns, K, sy);
    count_launch();
    return e;
}

// whether the persistent kernel takes this grid; sms set
bool rows_p_shape(const Dims &d, int &sms) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return false;
    sms = (dev >= 0 && dev < 64) ? g_sms[dev] : 0;
    return sms > 0 && d.nx % 64 == 0 && d.nx <= kPersMaxNx && d.ny >= kPersR;
}
// ... and these arrays (16-byte aligned for the copies)
bool rows_p_ok(const Dims &d, const void *a, const void *b, const void *c, int &sms) {
    const bool aligned = (((uintptr_t)a | (uintptr_t)b | (uintptr_t)c) & 15) == 0;
    return rows_p_shape(d, sms) && aligned;
}

}  // namespace

cudaError_t smoother_init() {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev >= 0 && dev < 64) {
        e = cudaDeviceGetAttribute(&g_sms[dev], cudaDevAttrMultiProcessorCount, dev);
        if (e != cudaSuccess) return e;
    }
    const int smem = (int)rows_smem(kRowsMaxThreads);
    const int smem_p = (int)(pers_floats(kPersMaxNx) * sizeof(float));
#define SET(kern, bytes)                                                                   \
    if ((e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes)) != \
        cudaSuccess)                                                                       \
        return e;
    SET((k_gs_rows<kRowsTY, 0, false>), smem)
    SET((k_gs_rows<kRowsTY, 0, true>), smem)
    SET((k_gs_rows<kRowsTY, 1, false>), smem)
    SET((k_gs_rows<kRowsTY, 1, true>), smem)
    SET((k_gs_rows_p<FineRowsOp, 0, false, false>), smem_p)
    SET((k_gs_rows_p<FineRowsOp, 0, true, false>), smem_p)
    SET((k_gs_rows_p<FineRowsOp, 1, false, false>), smem_p)
    SET((k_gs_rows_p<FineRowsOp, 1, true, false>), smem_p)
    SET((k_gs_rows_p<FineRowsOp, 0, false, true>), smem_p)
    SET((k_gs_rows_p<FineRowsOp, 0, true, true>), smem_p)
    SET((k_gs_rows_p<FineRowsOp, 1, false, true, true>), smem_p)
    SET((k_gs_rows_p<FineRowsOp, 1, true, true, true>), smem_p)
    SET((k_gs_rows_p<CoarseRowsOp, 0, false, false>), smem_p)
    SET((k_gs_rows_p<CoarseRowsOp, 1, false, false>), smem_p)
    const int smem_f = smem_p;
    SET((k_gs_rows_f<0, false>), smem_f)
    SET((k_gs_rows_f<0, true>), smem_f)
    SET((k_gs_rows_f<1, false>), smem_f)
    SET((k_gs_rows_f<1, true>), smem_f)
#undef SET
    // co-resident CTAs of the fused kernel for each row length it takes
    if (dev >= 0 && dev < 64)
        for (int w = 1; w <= kPersMaxNx / 64; w++) {
            const int nx = 64 * w;
            int lo = 1 << 30;
            const void *kerns[4] = {(const void *)k_gs_rows_f<0, false>,
                                    (const void *)k_gs_rows_f<0, true>,
                                    (const void *)k_gs_rows_f<1, false>,
                                    (const void *)k_gs_rows_f<1, true>};
            for (const void *kf : kerns) {
                int nb = 0;
                e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(
                    &nb, kf, nx / 2, pers_floats(nx) * sizeof(float));
                if (e != cudaSuccess) return e;
                lo = nb < lo ? nb : lo;
            }
            g_fused_slots[dev][w - 1] = lo * g_sms[dev];
        }
    return cudaSuccess;
}

bool fused_sweep_sizes(const Dims &d, long &naflag) {
    int sms = 0, dev = 0;
    if (!rows_p_shape(d, sms) || cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64)
        return false;
    if (fused_k(d, g_fused_slots[dev][d.nx / 64 - 1]) < 1) return false;
    naflag = (long)fused_nstrips(d) * (d.nz / 2 + 1);
    return true;
}

// one 8-colour sweep vin -> vout with the row-strip kernels, or
// cudaErrorNotSupported if the rows are too long for them
cudaError_t gs_sweep_fine_rows(const Dims &d, const Fine<float> &f, const float *b,
                               const float *vin, float *vout, bool descending, cudaStream_t s,
                               int split, const SweepSync *sync) {
    int sms = 0;
    if (rows_p_ok(d, b, vin, vout, sms)) {
        const FineRowsOp op{f};
        int dev = 0;
        const int kz = sync && cudaGetDevice(&dev) == cudaSuccess && dev >= 0 && dev < 64
                           ? fused_k(d, g_fused_slots[dev][d.nx / 64 - 1])
                           : 0;
        if (kz > 0) {
            // ascending: A = even planes from 2 (colours 0-3, F = 0);
            // descending: A = odd planes from 1 (colours 7-4, F = 1)
            if (!descending)
                return split ? launch_fused<0, true>(d, op, b, vin, vout, 2, kz, *sync, s)
                             : launch_fused<0, false>(d, op, b, vin, vout, 2, kz, *sync, s);
            return split ? launch_fused<1, true>(d, op, b, vin, vout, 1, kz, *sync, s)
                         : launch_fused<1, false>(d, op, b, vin, vout, 1, kz, *sync, s);
        }
        return split ? rows_p_sweep<FineRowsOp, true>(d, op, b, vin, vout, descending, s, sms)
                     : rows_p_sweep<FineRowsOp, false>(d, op, b, vin, vout, descending, s, sms);
    }
    if (d.nx / 2 > kRowsMaxThreads) return cudaErrorNotSupported;
    cudaError_t e;
    if (!descending) {
        e = rows_phase<0>(d, f, b, vin, vin, vout, 0, s, split);
        if (e != cudaSuccess) return e;
        return rows_phase<0>(d, f, b, vin, vout, vout, 1, s, split);
    }
    e = rows_phase<1>(d, f, b, vin, vin, vout, 1, s, split);
    if (e != cudaSuccess) return e;
    return rows_phase<1>(d, f, b, vin, vout, vout, 0, s, split);
}

// FP32 finest-level residual r = b - A x (interior planes) with the
// persistent row-strip kernel, or cudaErrorNotSupported
cudaError_t residual_fine_rows(const Dims &d, const Fine<float> &f, const float *b,
                               const float *x, float *r, cudaStream_t s, int split) {
    int sms = 0;
    if (!rows_p_ok(d, b, x, r, sms)) return cudaErrorNotSupported;
    const FineRowsOp op{f};
    return split ? launch_rows_p<FineRowsOp, 0, true, true>(d, op, b, x, x, r, 1, 1, d.nz - 1, s,
                                                            sms)
                 : launch_rows_p<FineRowsOp, 0, false, true>(d, op, b, x, x, r, 1, 1, d.nz - 1,
                                                             s, sms);
}

// The finest FP32 residual restricted to the next level without storing it
// (rows as residual_fine_rows; ny even and nz >= 4 even): the residual
// kernel writes the x-y restricted partial sums of every fine plane into
// part (3 (nz+1) ny/2 nx/2 floats), k_restrict_z combines them along z into
// bc; or cudaErrorNotSupported.
cudaError_t residual_restrict_fine_rows(const Dims &d, const Fine<float> &f, const float *b,
                                        const float *x, float *part, float *bc, cudaStream_t s,
                                        int split) {
    int sms = 0;
    static_assert(kPersTY % 2 == 0, "coarse rows of a strip need an even strip height");
    if ((d.ny & 1) || d.nz < 4 || (d.nz & 1) || !rows_p_ok(d, b, x, part, sms))
        return cudaErrorNotSupported;
    const FineRowsOp op{f};
    const cudaError_t e =
        split ? launch_rows_p<FineRowsOp, 1, true, true, true>(d, op, b, x, x, part, 1, 1,
                                                                d.nz - 1, s, sms)
              : launch_rows_p<FineRowsOp, 1, false, true, true>(d, op, b, x, x, part, 1, 1,
                                                                 d.nz - 1, s, sms);
    if (e != cudaSuccess) return e;
    return restrict_z(d, part, bc, s);
}

// Coarse levels take the row strips only where they win (measured on GB300,
// 27-point stencil, FMA-issue bound in every form): rows of 128 nodes and up
// (128^3 level: 98 us a sweep against 103 us for eight colour launches); at
// 64^3 the tile kernel is faster (35 against 49 us), and the coarse residual
// stays one thread per node (55 against 59 us at 128^3).
bool coarse_rows_fit(const Dims &d) {
    int sms = 0;
    return d.nx >= 128 && rows_p_shape(d, sms);
}

// coarse-level FP32 sweep with the persistent row-strip kernel (natural
// column order), or cudaErrorNotSupported
cudaError_t gs_sweep_coarse_rows(const Dims &d, const Coarse<float> &c, const float *b,
                                 const float *vin, float *vout, bool descending, cudaStream_t s) {
    int sms = 0;
    if (d.nx < 128 || !rows_p_ok(d, b, vin, vout, sms)) return cudaErrorNotSupported;
    const CoarseRowsOp op{c};
    return rows_p_sweep<CoarseRowsOp, false>(d, op, b, vin, vout, descending, s, sms);
}

}  // namespace qsmg

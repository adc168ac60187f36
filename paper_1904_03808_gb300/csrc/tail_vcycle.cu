// tail_vcycle.cu -- the bottom of the FP32 V-cycle in one thread block.
//
// Below some level every array of the hierarchy fits in one SM's shared
// memory (typically 16^3 -> 8^3 -> 4^3 cells).  There the V-cycle of section
// 3.6 is pure launch latency when each colour pass, residual, restriction and
// prolongation is its own kernel, so this kernel runs all of it -- 8-colour
// Gauss-Seidel sweeps, residual, full-weighting restriction, the dense
// coarsest solve, trilinear prolongation -- inside one 512-thread block with
// block barriers between the passes.  Every pass uses the same arithmetic, in
// the same order per node, as the corresponding multi-kernel pass.
#include "qsmg_impl.h"

namespace qsmg {
namespace {

constexpr int NT = 512;

struct Lev {
    int nx, ny, nz;
    int cs;   // component stride (nz+1)*ny*nx
    int off;  // shared-memory word offset of this level's x, then b, then r
};

__device__ __forceinline__ int wrapi(int i, int n) { return i < 0 ? i + n : (i >= n ? i - n : i); }

// the stencil pointer passed through an opaque move: its 243 coefficients
// are then re-read (read-only cache broadcasts) instead of being hoisted into
// registers, which would spill
__device__ __forceinline__ const float *opaque(const float *p) {
    const float *q;
    asm volatile("mov.b64 %0, %1;" : "=l"(q) : "l"(p));
    return q;
}

// one colour pass on level L (27-point stencil S, centre inverse Dinv)
__device__ void colour(const Lev &L, float *x, const float *b, const float *__restrict__ S0,
                       const float *__restrict__ Dinv, int colour) {
    const int hx = L.nx / 2, hy = L.ny / 2;
    const int nk = (colour & 4) ? L.nz / 2 : L.nz / 2 - 1;
    const int tot = hx * hy * nk;
    for (int t = threadIdx.x; t < tot; t += NT) {
        const int ix = t % hx, q = t / hx, jy = q % hy, kz = q / hy;
        const int i = 2 * ix + (colour & 1), j = 2 * jy + ((colour >> 1) & 1);
        const int k = 2 * kz + ((colour & 4) ? 1 : 2);
        const float *S = opaque(S0);
        float s0 = 0.f, s1 = 0.f, s2 = 0.f;
#pragma unroll
        for (int dz = -1; dz <= 1; dz++)
#pragma unroll
            for (int dy = -1; dy <= 1; dy++) {
                const int row = ((k + dz) * L.ny + wrapi(j + dy, L.ny)) * L.nx;
#pragma unroll
                for (int dx = -1; dx <= 1; dx++) {
                    const int dd = (dz + 1) * 9 + (dy + 1) * 3 + (dx + 1);
                    if (dd == 13) continue;
                    const int q2 = row + wrapi(i + dx, L.nx);
                    const float v0 = x[q2], v1 = x[q2 + L.cs], v2 = x[q2 + 2 * L.cs];
                    const float *s = S + dd * 9;
                    s0 += __ldg(s) * v0 + __ldg(s + 1) * v1 + __ldg(s + 2) * v2;
                    s1 += __ldg(s + 3) * v0 + __ldg(s + 4) * v1 + __ldg(s + 5) * v2;
                    s2 += __ldg(s + 6) * v0 + __ldg(s + 7) * v1 + __ldg(s + 8) * v2;
                }
            }
        const int p = (k * L.ny + j) * L.nx + i;
        const float f0 = b[p] - s0, f1 = b[p + L.cs] - s1, f2 = b[p + 2 * L.cs] - s2;
        x[p] = Dinv[0] * f0 + Dinv[1] * f1 + Dinv[2] * f2;
        x[p + L.cs] = Dinv[3] * f0 + Dinv[4] * f1 + Dinv[5] * f2;
        x[p + 2 * L.cs] = Dinv[6] * f0 + Dinv[7] * f1 + Dinv[8] * f2;
    }
}

__device__ void sweeps(const Lev &L, float *x, const float *b, const float *S, const float *Dinv,
                       int n, bool descending) {
    for (int s = 0; s < n; s++)
        for (int c = 0; c < 8; c++) {
            colour(L, x, b, S, Dinv, descending ? 7 - c : c);
            __syncthreads();
        }
}

// r = b - A x on interior nodes (walls of r unused)
__device__ void residual(const Lev &L, const float *x, const float *b, float *r,
                         const float *__restrict__ S0) {
    const int tot = L.nx * L.ny * (L.nz - 1);
    for (int t = threadIdx.x; t < tot; t += NT) {
        const int i = t % L.nx, q = t / L.nx, j = q % L.ny, k = q / L.ny + 1;
        const float *S = opaque(S0);
        float s0 = 0.f, s1 = 0.f, s2 = 0.f;
#pragma unroll
        for (int dz = -1; dz <= 1; dz++)
#pragma unroll
            for (int dy = -1; dy <= 1; dy++) {
                const int row = ((k + dz) * L.ny + wrapi(j + dy, L.ny)) * L.nx;
#pragma unroll
                for (int dx = -1; dx <= 1; dx++) {
                    const int dd = (dz + 1) * 9 + (dy + 1) * 3 + (dx + 1);
                    if (dd == 13) continue;
                    const int q2 = row + wrapi(i + dx, L.nx);
                    const float v0 = x[q2], v1 = x[q2 + L.cs], v2 = x[q2 + 2 * L.cs];
                    const float *s = S + dd * 9;
                    s0 += __ldg(s) * v0 + __ldg(s + 1) * v1 + __ldg(s + 2) * v2;
                    s1 += __ldg(s + 3) * v0 + __ldg(s + 4) * v1 + __ldg(s + 5) * v2;
                    s2 += __ldg(s + 6) * v0 + __ldg(s + 7) * v1 + __ldg(s + 8) * v2;
                }
            }
        const int p = (k * L.ny + j) * L.nx + i;
        const float x0 = x[p], x1 = x[p + L.cs], x2 = x[p + 2 * L.cs];
        const float *c = S + 13 * 9;
        r[p] = b[p] - (s0 + __ldg(c) * x0 + __ldg(c + 1) * x1 + __ldg(c + 2) * x2);
        r[p + L.cs] = b[p + L.cs] - (s1 + __ldg(c + 3) * x0 + __ldg(c + 4) * x1 + __ldg(c + 5) * x2);
        r[p + 2 * L.cs] =
            b[p + 2 * L.cs] - (s2 + __ldg(c + 6) * x0 + __ldg(c + 7) * x1 + __ldg(c + 8) * x2);
    }
}

// bc = T^T r (coarse interior), coarse walls zero
__device__ void restrict_to(const Lev &F, const Lev &C, const float *r, float *bc) {
    const int tot = C.nx * C.ny * (C.nz + 1);
    for (int t = threadIdx.x; t < tot; t += NT) {
        const int I = t % C.nx, q = t / C.nx, J = q % C.ny, K = q / C.ny;
        const int p = (K * C.ny + J) * C.nx + I;
        if (K == 0 || K == C.nz) {
            bc[p] = bc[p + C.cs] = bc[p + 2 * C.cs] = 0.f;
            continue;
        }
        float s0 = 0.f, s1 = 0.f, s2 = 0.f;
#pragma unroll
        for (int ez = -1; ez <= 1; ez++) {
            const float wz = ez ? 0.5f : 1.f;
            const int pl = (2 * K + ez) * F.ny;
#pragma unroll
            for (int ey = -1; ey <= 1; ey++) {
                const float wy = ey ? 0.5f : 1.f;
                const int row = (pl + wrapi(2 * J + ey, F.ny)) * F.nx;
#pragma unroll
                for (int ex = -1; ex <= 1; ex++) {
                    const float w = (ex ? 0.5f : 1.f) * wy * wz;
                    const int q2 = row + wrapi(2 * I + ex, F.nx);
                    s0 += w * r[q2];
                    s1 += w * r[q2 + F.cs];
                    s2 += w * r[q2 + 2 * F.cs];
                }
            }
        }
        bc[p] = s0;
        bc[p + C.cs] = s1;
        bc[p + 2 * C.cs] = s2;
    }
}

// x += T xc on fine interior nodes (coarse walls are zero)
__device__ void prolong_to(const Lev &F, const Lev &C, const float *xc, float *x) {
    const int tot = F.nx * F.ny * (F.nz - 1);
    for (int t = threadIdx.x; t < tot; t += NT) {
        const int i = t % F.nx, q = t / F.nx, j = q % F.ny, k = q / F.ny + 1;
        const int I0 = i >> 1, J0 = j >> 1, K0 = k >> 1;
        const int I1 = (i & 1) ? ((I0 + 1 < C.nx) ? I0 + 1 : 0) : I0;
        const int J1 = (j & 1) ? ((J0 + 1 < C.ny) ? J0 + 1 : 0) : J0;
        const int K1 = (k & 1) ? K0 + 1 : K0;
        const float wx = (i & 1) ? 0.5f : 1.f, wy = (j & 1) ? 0.5f : 1.f, wz = (k & 1) ? 0.5f : 1.f;
        const int ni = (i & 1) ? 2 : 1, nj = (j & 1) ? 2 : 1, nk = (k & 1) ? 2 : 1;
        const int Is[2] = {I0, I1}, Js[2] = {J0, J1}, Ks[2] = {K0, K1};
        const int p = (k * F.ny + j) * F.nx + i;
#pragma unroll
        for (int a = 0; a < 3; a++) {
            float s = 0.f;
            for (int u = 0; u < nk; u++)
                for (int v = 0; v < nj; v++)
                    for (int w = 0; w < ni; w++)
                        s += xc[a * C.cs + (Ks[u] * C.ny + Js[v]) * C.nx + Is[w]];
            x[p + a * F.cs] += wx * wy * wz * s;
        }
    }
}

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    return v;
}

template <int NLEV>
struct TailArgs {
    Lev lev[NLEV];
    const float *S[NLEV];     // device copies of the level stencils (243 + 9 floats)
    const double *Ainv;       // dense inverse of the coarsest operator
    int ncoarse, nu1, nu2, nlev;
};

constexpr int kMaxTail = 6;

__global__ void __launch_bounds__(NT, 1)
    k_tail_vcycle(TailArgs<kMaxTail> A, const float *__restrict__ bg, float *__restrict__ xg) {
    extern __shared__ __align__(16) float sm[];
    __shared__ Lev lev[kMaxTail];
    __shared__ const float *Sp[kMaxTail];
    const int nl = A.nlev;
    if (threadIdx.x < kMaxTail) {
        lev[threadIdx.x] = A.lev[threadIdx.x];
        Sp[threadIdx.x] = A.S[threadIdx.x];
    }
    __syncthreads();
    // load the top tail level's x and b
    {
        const Lev &T = lev[0];
        const int n = 3 * T.cs;
        for (int t = threadIdx.x; t < n; t += NT) {
            sm[T.off + t] = xg[t];
            sm[T.off + n + t] = bg[t];
        }
    }
    __syncthreads();
    // down: smooth, residual, restrict, zero the coarse iterate
    for (int l = 0; l < nl - 1; l++) {
        const Lev &L = lev[l], &C = lev[l + 1];
        float *x = sm + L.off, *b = x + 3 * L.cs, *r = b + 3 * L.cs;
        sweeps(L, x, b, Sp[l], Sp[l] + 243, A.nu1, false);
        residual(L, x, b, r, Sp[l]);
        __syncthreads();
        float *xc = sm + C.off, *bcv = xc + 3 * C.cs;
        restrict_to(L, C, r, bcv);
        for (int t = threadIdx.x; t < 3 * C.cs; t += NT) xc[t] = 0.f;
        __syncthreads();
    }
    // coarsest: x = Ainv b (x starts at zero with zero walls); one warp a row
    {
        const Lev &C = lev[nl - 1];
        float *x = sm + C.off, *b = x + 3 * C.cs;
        const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
        const int plane0 = C.ny * C.nx;
        for (int row = warp; row < A.ncoarse; row += NT / 32) {
            double acc = 0.0;
            for (int v = lane; v < A.ncoarse; v += 32)
                acc += A.Ainv[(long)row * A.ncoarse + v] * (double)b[(v % 3) * C.cs + plane0 + v / 3];
            acc = warp_sum(acc);
            if (lane == 0) {
                const int p = (row % 3) * C.cs + plane0 + row / 3;
                x[p] = (float)((double)x[p] + acc);
            }
        }
    }
    __syncthreads();
    // up: prolongate and post-smooth
    for (int l = nl - 2; l >= 0; l--) {
        const Lev &L = lev[l], &C = lev[l + 1];
        float *x = sm + L.off, *b = x + 3 * L.cs;
        prolong_to(L, C, sm + C.off, x);
        __syncthreads();
        sweeps(L, x, b, Sp[l], Sp[l] + 243, A.nu2, true);
    }
    // store the top tail level's x
    {
        const Lev &T = lev[0];
        for (int t = threadIdx.x; t < 3 * T.cs; t += NT) xg[t] = sm[T.off + t];
    }
}

}  // namespace

size_t tail_smem_bytes(const int dims[][3], int nlev) {
    size_t words = 0;
    for (int l = 0; l < nlev; l++) {
        const size_t cs = (size_t)(dims[l][2] + 1) * dims[l][1] * dims[l][0];
        words += (l + 1 < nlev ? 3 : 2) * 3 * cs;  // x, b (and r above the coarsest)
    }
    return words * sizeof(float);
}

cudaError_t tail_vcycle(const int dims[][3], int nlev, const float *const *S, const double *Ainv,
                        int ncoarse, int nu1, int nu2, const float *b, float *x,
                        cudaStream_t s) {
    if (nlev < 2 || nlev > kMaxTail) return cudaErrorInvalidValue;
    TailArgs<kMaxTail> A;
    int off = 0;
    for (int l = 0; l < nlev; l++) {
        A.lev[l].nx = dims[l][0];
        A.lev[l].ny = dims[l][1];
        A.lev[l].nz = dims[l][2];
        A.lev[l].cs = (dims[l][2] + 1) * dims[l][1] * dims[l][0];
        A.lev[l].off = off;
        off += (l + 1 < nlev ? 3 : 2) * 3 * A.lev[l].cs;
        A.S[l] = S[l];
    }
    A.Ainv = Ainv;
    A.ncoarse = ncoarse;
    A.nu1 = nu1;
    A.nu2 = nu2;
    A.nlev = nlev;
    const size_t smem = (size_t)off * sizeof(float);
    cudaError_t e = cudaFuncSetAttribute(k_tail_vcycle, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
    k_tail_vcycle<<<1, NT, smem, s>>>(A, b, x);
    count_launch();
    return cudaGetLastError();
}

}  // namespace qsmg

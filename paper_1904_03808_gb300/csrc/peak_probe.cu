// peak_probe.cu -- a measurement aid, separate from the method's library: the
// fused multiply-add rate this GPU sustains in FP64 and in FP32, the
// denominator of the roofline of the FP64 pointwise kernels (GB300 runs FP64
// arithmetic at a small fraction of its FP32 rate, so those kernels are
// bound by the FP64 pipe rather than by HBM).
//
// Every thread runs CH independent chains x <- x * a + b for iters rounds, so
// the pipe always has independent work; a and b arrive as arguments and every
// thread stores its chains' sum, so nothing can be folded away.  One launch
// does 2 * CH * iters flops a thread.
#include <cuda_runtime.h>

namespace {

constexpr int CH = 16;
constexpr int kThreads = 256;

template <class T>
__global__ void __launch_bounds__(kThreads) k_fma_chains(T *__restrict__ out, int iters, T a, T b) {
    T x[CH];
#pragma unroll
    for (int c = 0; c < CH; c++) x[c] = (T)(threadIdx.x + c) * (T)1e-3;
    for (int i = 0; i < iters; i++) {
#pragma unroll
        for (int c = 0; c < CH; c++) x[c] = fma(x[c], a, b);
    }
    T s = 0;
#pragma unroll
    for (int c = 0; c < CH; c++) s += x[c];
    out[(long)blockIdx.x * kThreads + threadIdx.x] = s;
}

template <class T>
int run(int blocks_per_sm, int iters, int reps, double *tflops, double *ms) {
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 1;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 1;
    const int blocks = sms * blocks_per_sm;
    T *out = nullptr;
    if (cudaMalloc(&out, sizeof(T) * (size_t)blocks * kThreads) != cudaSuccess) return 2;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    const T a = (T)0.999999, b = (T)1e-7;
    k_fma_chains<T><<<blocks, kThreads>>>(out, iters / 10 + 1, a, b);  // warm-up
    float best = 0.f;
    for (int r = 0; r < reps; r++) {
        cudaEventRecord(e0);
        k_fma_chains<T><<<blocks, kThreads>>>(out, iters, a, b);
        cudaEventRecord(e1);
        cudaEventSynchronize(e1);
        float t = 0.f;
        cudaEventElapsedTime(&t, e0, e1);
        if (r == 0 || t < best) best = t;
    }
    const cudaError_t err = cudaGetLastError();
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(out);
    if (err != cudaSuccess) return 3;
    const double flops = 2.0 * CH * (double)iters * (double)blocks * kThreads;
    *ms = best;
    *tflops = flops / (best * 1e-3) / 1e12;
    return 0;
}

}  // namespace

// fp64 != 0: FP64 chains, else FP32.  blocks_per_sm CTAs of 256 threads on
// every SM, iters rounds of CH chains, reps timed launches (the fastest is
// kept).  Returns 0, or 1 (no device), 2 (allocation), 3 (launch) failure.
extern "C" int qsmg_fma_peak(int fp64, int blocks_per_sm, int iters, int reps, double *tflops,
                             double *ms) {
    if (!tflops || !ms || blocks_per_sm < 1 || iters < 1 || reps < 1) return 4;
    return fp64 ? run<double>(blocks_per_sm, iters, reps, tflops, ms)
                : run<float>(blocks_per_sm, iters, reps, tflops, ms);
}

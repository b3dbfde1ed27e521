// ibf_probe.cu -- throughput of the fp64 pipe (libibf_probe.so), the denominator of the
// fp64 projection path's roofline: that path's transforms and sweeps run on the fp64
// pipe, whose rate is not among the copy-bandwidth and bf16 GEMM peaks measured for the
// device.  Not part of the projection library.
//
// Each thread runs kChains independent dependent-free chains of fp64 FMAs (or adds) for
// `iters` steps; the grid is 8 CTAs of 256 threads per SM, so every SM has enough warps
// in flight to hide the pipe's latency.  The chains' sums are written out so that the
// compiler keeps the arithmetic.
#include <cuda_runtime.h>

namespace {

constexpr int kChains = 8;
constexpr int kThreads = 256;

template <bool FMA>
__global__ void __launch_bounds__(kThreads) k_fp64_chains(double *out, int iters, double b, double c) {
    double a[kChains];
#pragma unroll
    for (int i = 0; i < kChains; ++i) a[i] = (double)(threadIdx.x + i);
    for (int t = 0; t < iters; ++t) {
#pragma unroll
        for (int i = 0; i < kChains; ++i) a[i] = FMA ? fma(a[i], b, c) : a[i] + c;
    }
    double s = 0.0;
#pragma unroll
    for (int i = 0; i < kChains; ++i) s += a[i];
    out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

template <bool FMA>
int time_chains(int nblk, double *buf, int iters, double *gops) {
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess) return 1;
    if (cudaEventCreate(&e1) != cudaSuccess) { cudaEventDestroy(e0); return 1; }
    // b slightly below 1 and c small keep every value finite and normal
    k_fp64_chains<FMA><<<nblk, kThreads>>>(buf, iters, 0.999999, 1e-7);  // warm-up
    cudaEventRecord(e0);
    k_fp64_chains<FMA><<<nblk, kThreads>>>(buf, iters, 0.999999, 1e-7);
    cudaEventRecord(e1);
    int rc = cudaEventSynchronize(e1) == cudaSuccess ? 0 : 1;
    float ms = 0.f;
    if (!rc) rc = cudaEventElapsedTime(&ms, e0, e1) == cudaSuccess ? 0 : 1;
    if (!rc) *gops = (double)nblk * kThreads * (double)iters * kChains / (ms * 1e-3) / 1e9;
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return rc;
}

}  // namespace

// Measures the fp64 FMA and add instruction rates of the current device in Gop/s (one
// FMA or add per operation; an FMA counts as two flops).  Returns 0 on success, 1 if a
// CUDA call failed.  Allocates and frees a small output buffer; synchronises the device.
extern "C" int ibfprobe_fp64_rates(double *dfma_gops, double *dadd_gops) {
    int dev = 0, nsm = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 1;
    if (cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 1;
    const int nblk = 8 * nsm;
    double *buf = nullptr;
    if (cudaMalloc(&buf, (size_t)nblk * kThreads * sizeof(double)) != cudaSuccess) return 1;
    const int iters = 1 << 14;
    int rc = time_chains<true>(nblk, buf, iters, dfma_gops);
    if (!rc) rc = time_chains<false>(nblk, buf, iters, dadd_gops);
    cudaFree(buf);
    (void)cudaGetLastError();
    return rc;
}

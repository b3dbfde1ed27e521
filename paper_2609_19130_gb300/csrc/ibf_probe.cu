// ibf_probe.cu -- instruction throughput probes (libibf_probe.so).  The fp64 rates are
// the denominator of the fp64 projection path's roofline: that path's transforms and
// sweeps run on the fp64 pipe, whose rate is not among the copy-bandwidth and bf16 GEMM
// peaks measured for the device.  The other rates (fp32 FMA, conversions between fp64 and
// fp32, integer-to-float conversion, 32-bit integer add and logic) are the facts behind
// the mixed path's choice of float-float arithmetic with integer-based conversions.  Not
// part of the projection library.
//
// Each thread runs kChains independent chains of one operation (or one fixed pair of
// operations) for `iters` steps; the grid is 8 CTAs of 256 threads per SM, so every SM
// has enough warps in flight to hide the pipe's latency.  The chains' final values are
// written out so that the compiler keeps the arithmetic.
#include <cuda_runtime.h>

namespace {

constexpr int kChains = 8;
constexpr int kThreads = 256;

// operation kinds, in the order of ibfprobe_op_rates' output
enum Op { OP_DFMA = 0, OP_DADD, OP_FFMA, OP_F2F_PAIR, OP_I2F_PAIR, OP_INT_PAIR, OP_COUNT };

template <int OP>
__global__ void __launch_bounds__(kThreads) k_chains(double *out, int iters, double b, double c) {
    if constexpr (OP == OP_DFMA || OP == OP_DADD) {
        double a[kChains];
#pragma unroll
        for (int i = 0; i < kChains; ++i) a[i] = (double)(threadIdx.x + i);
        for (int t = 0; t < iters; ++t) {
#pragma unroll
            for (int i = 0; i < kChains; ++i) a[i] = OP == OP_DFMA ? fma(a[i], b, c) : a[i] + c;
        }
        double s = 0.0;
#pragma unroll
        for (int i = 0; i < kChains; ++i) s += a[i];
        out[blockIdx.x * blockDim.x + threadIdx.x] = s;
    } else if constexpr (OP == OP_FFMA) {
        const float bf = (float)b, cf = (float)c;
        float a[kChains];
#pragma unroll
        for (int i = 0; i < kChains; ++i) a[i] = (float)(threadIdx.x + i);
        for (int t = 0; t < iters; ++t) {
#pragma unroll
            for (int i = 0; i < kChains; ++i) a[i] = __fmaf_rn(a[i], bf, cf);
        }
        float s = 0.f;
#pragma unroll
        for (int i = 0; i < kChains; ++i) s += a[i];
        out[blockIdx.x * blockDim.x + threadIdx.x] = s;
    } else if constexpr (OP == OP_F2F_PAIR) {
        // fp64 -> fp32 (round to nearest) -> fp64: two conversions a step
        double a[kChains];
#pragma unroll
        for (int i = 0; i < kChains; ++i) a[i] = (double)(threadIdx.x + i) * c;
        for (int t = 0; t < iters; ++t) {
#pragma unroll
            for (int i = 0; i < kChains; ++i) a[i] = (double)__double2float_rn(a[i]);
        }
        double s = 0.0;
#pragma unroll
        for (int i = 0; i < kChains; ++i) s += a[i];
        out[blockIdx.x * blockDim.x + threadIdx.x] = s;
    } else if constexpr (OP == OP_I2F_PAIR) {
        // u32 -> fp32 conversion, then its bit pattern xor a constant: one I2F and one
        // logic op a step
        unsigned a[kChains];
#pragma unroll
        for (int i = 0; i < kChains; ++i) a[i] = threadIdx.x * 7u + i;
        const unsigned m = 0x5A5A5u;
        for (int t = 0; t < iters; ++t) {
#pragma unroll
            for (int i = 0; i < kChains; ++i) a[i] = __float_as_uint(__uint2float_rn(a[i])) ^ m;
        }
        unsigned s = 0u;
#pragma unroll
        for (int i = 0; i < kChains; ++i) s += a[i];
        out[blockIdx.x * blockDim.x + threadIdx.x] = (double)s;
    } else {
        // 32-bit integer add then xor: two integer ops a step
        unsigned a[kChains];
#pragma unroll
        for (int i = 0; i < kChains; ++i) a[i] = threadIdx.x * 7u + i;
        const unsigned m = 0x5A5A5u, d = 0x9E3779B9u + blockIdx.x;
        for (int t = 0; t < iters; ++t) {
#pragma unroll
            for (int i = 0; i < kChains; ++i) a[i] = (a[i] + d) ^ m;
        }
        unsigned s = 0u;
#pragma unroll
        for (int i = 0; i < kChains; ++i) s += a[i];
        out[blockIdx.x * blockDim.x + threadIdx.x] = (double)s;
    }
}

// steps a thread executes per chain step: two for the pairs
constexpr double kOpsPerStep[OP_COUNT] = {1, 1, 1, 2, 2, 2};

template <int OP>
int time_chains(int nblk, double *buf, int iters, double *gops) {
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess) return 1;
    if (cudaEventCreate(&e1) != cudaSuccess) { cudaEventDestroy(e0); return 1; }
    // b slightly below 1 and c small keep every value finite and normal
    k_chains<OP><<<nblk, kThreads>>>(buf, iters, 0.999999, 1e-7);  // warm-up
    cudaEventRecord(e0);
    k_chains<OP><<<nblk, kThreads>>>(buf, iters, 0.999999, 1e-7);
    cudaEventRecord(e1);
    int rc = cudaEventSynchronize(e1) == cudaSuccess ? 0 : 1;
    float ms = 0.f;
    if (!rc) rc = cudaEventElapsedTime(&ms, e0, e1) == cudaSuccess ? 0 : 1;
    if (!rc) *gops = (double)nblk * kThreads * (double)iters * kChains * kOpsPerStep[OP] / (ms * 1e-3) / 1e9;
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return rc;
}

int probe(int nops, double *gops) {
    int dev = 0, nsm = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 1;
    if (cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 1;
    const int nblk = 8 * nsm;
    double *buf = nullptr;
    if (cudaMalloc(&buf, (size_t)nblk * kThreads * sizeof(double)) != cudaSuccess) return 1;
    const int iters = 1 << 14;
    int rc = 0;
    if (!rc && nops > OP_DFMA) rc = time_chains<OP_DFMA>(nblk, buf, iters, gops + OP_DFMA);
    if (!rc && nops > OP_DADD) rc = time_chains<OP_DADD>(nblk, buf, iters, gops + OP_DADD);
    if (!rc && nops > OP_FFMA) rc = time_chains<OP_FFMA>(nblk, buf, iters, gops + OP_FFMA);
    if (!rc && nops > OP_F2F_PAIR) rc = time_chains<OP_F2F_PAIR>(nblk, buf, iters, gops + OP_F2F_PAIR);
    if (!rc && nops > OP_I2F_PAIR) rc = time_chains<OP_I2F_PAIR>(nblk, buf, iters, gops + OP_I2F_PAIR);
    if (!rc && nops > OP_INT_PAIR) rc = time_chains<OP_INT_PAIR>(nblk, buf, iters, gops + OP_INT_PAIR);
    cudaFree(buf);
    (void)cudaGetLastError();
    return rc;
}

}  // namespace

// Measures the fp64 FMA and add instruction rates of the current device in Gop/s (one
// FMA or add per operation; an FMA counts as two flops).  Returns 0 on success, 1 if a
// CUDA call failed.  Allocates and frees a small output buffer; synchronises the device.
extern "C" int ibfprobe_fp64_rates(double *dfma_gops, double *dadd_gops) {
    double g[2] = {0.0, 0.0};
    const int rc = probe(2, g);
    *dfma_gops = g[0];
    *dadd_gops = g[1];
    return rc;
}

// Measures, in Gop/s (instructions of the named kind per second, device-wide), the first
// min(n, 6) of: fp64 FMA, fp64 add, fp32 FMA, fp64<->fp32 conversion (a round trip, two
// conversions per step), u32->fp32 conversion paired with one xor, 32-bit integer add
// paired with one xor.  For the pairs the rate counts both instructions.  Returns 0 on
// success, 1 if a CUDA call failed; synchronises the device.
extern "C" int ibfprobe_op_rates(double *gops, int n) {
    for (int i = 0; i < n; ++i) gops[i] = 0.0;
    return probe(n < OP_COUNT ? n : OP_COUNT, gops);
}

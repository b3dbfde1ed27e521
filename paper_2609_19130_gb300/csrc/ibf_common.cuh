// ibf_common.cuh -- device helpers shared by the x-direction kernels (ibf_kernels.cu)
// and the y/z-direction kernels (ibf_yz.cu): grid lookup of batched launches,
// precision-policy traits, fixed-order block reductions, warp shuffles, phi sources
// and the row-segment mapping of the x kernels.
#pragma once
#include "ibf_device.cuh"
#include "ibf_internal.h"

namespace ibf {

__device__ __forceinline__ int find_grid(const int *start, int n, int b) {
    int lo = 0, hi = n;  // start[lo] <= b < start[hi]
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (__ldg(start + mid) <= b) lo = mid; else hi = mid;
    }
    return lo;
}

// cp.async (sm_80+ asynchronous global->shared copy, L1-bypassing for 16 B) of one element
template <int BYTES> __device__ __forceinline__ void cp_async(void *smem_dst, const void *gmem_src) {
    const unsigned sa = (unsigned)__cvta_generic_to_shared(smem_dst);
    if constexpr (BYTES == 16)
        asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(sa), "l"(gmem_src));
    else
        asm volatile("cp.async.ca.shared.global [%0], [%1], %2;\n" ::"r"(sa), "l"(gmem_src), "n"(BYTES));
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::); }
template <int N> __device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N)); }

// Bulk asynchronous copies (sm_90+ cp.async.bulk, the copy engine behind TMA) of a
// contiguous global range into shared memory, completed on an mbarrier by byte count.
// Sources are this GPU's global memory; no cluster multicast is used.
__device__ __forceinline__ unsigned smem_u32(const void *p) { return (unsigned)__cvta_generic_to_shared(p); }
__device__ __forceinline__ void mbar_init(unsigned long long *bar, unsigned count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
// make the initialised barriers visible to the async proxy (the copy engine)
__device__ __forceinline__ void mbar_init_fence() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }
// one arrival that also announces `bytes` of copies completing on the barrier
__device__ __forceinline__ void mbar_arrive_expect_tx(unsigned long long *bar, unsigned bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(unsigned long long *bar, unsigned parity) {
    unsigned ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}
// Wait for phase `parity` of the barrier to complete, giving up after `limit` polls
// (each try_wait already suspends the thread for a while); returns false on giving up.
__device__ __forceinline__ bool mbar_wait_bounded(unsigned long long *bar, unsigned parity, unsigned limit) {
    for (unsigned it = 0; it < limit; ++it)
        if (mbar_try_wait(bar, parity)) return true;
    return false;
}
// global -> shared copy of `bytes` (a multiple of 16; both addresses 16-byte aligned)
__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, unsigned bytes, unsigned long long *bar) {
    asm volatile("cp.async.bulk.shared::cta.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     smem_u32(dst)),
                 "l"(src), "r"(bytes), "r"(smem_u32(bar))
                 : "memory");
}
// hint: bring `bytes` (a multiple of 16, 16-byte aligned source) of global memory into L2
__device__ __forceinline__ void bulk_prefetch_l2(const void *src, unsigned bytes) {
    asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(src), "r"(bytes) : "memory");
}
// order this thread's earlier shared-memory accesses before later async-proxy writes
__device__ __forceinline__ void fence_proxy_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
__device__ __forceinline__ void mbar_inval(unsigned long long *bar) {
    asm volatile("mbarrier.inval.shared::cta.b64 [%0];" ::"r"(smem_u32(bar)) : "memory");
}

template <class A> struct IsDF { static constexpr bool value = false; };
template <> struct IsDF<DFArith> { static constexpr bool value = true; };

template <class A> struct Coef;
template <> struct Coef<F64Arith> {
    __device__ __forceinline__ static double c(double x) { return x; }
    __device__ __forceinline__ static double c2(float2 v, double x) { return x; }
};
template <> struct Coef<DFArith> {
    // per-CTA constants: the general conversion, in line (no call in the kernel's prologue)
    __device__ __forceinline__ static df c(double x) { return f64_to_df_general(x); }
    __device__ __forceinline__ static df c2(float2 v, double) { return {v.x, v.y}; }
};

template <class A> __device__ __forceinline__ float absv(typename A::V v);
template <> __device__ __forceinline__ float absv<F64Arith>(double v) { return fabsf((float)v); }
template <> __device__ __forceinline__ float absv<DFArith>(df v) { return fabsf(v.hi); }

template <typename T, class A> __device__ __forceinline__ T to_T(typename A::V v);
template <> __device__ __forceinline__ double to_T<double, F64Arith>(double v) { return v; }
template <> __device__ __forceinline__ float to_T<float, DFArith>(df v) { return df_to_f(v); }

// DCT-II through an N-point FFT (Makhoul, IEEE TASSP 28(1), 1980): sample i goes to
// FFT input position i/2 (i even) or N - (i+1)/2 (i odd); the inverse un-reorders the
// same way.  Coefficient m is Re(exp(-i pi m/(2N)) V_m) of the FFT V of the reordered
// sequence.
__device__ __forceinline__ int dct_perm(int i, int n) { return (i & 1) ? n - ((i + 1) >> 1) : (i >> 1); }

// ---------------------------------------------------------------- block reductions (fixed order)
template <class A> struct Red;
template <> struct Red<F64Arith> {
    __device__ static double sum(double v, double *sh) {
        for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
        const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
        if (lane == 0) sh[wid] = v;
        __syncthreads();
        double r = 0.0;
        if (threadIdx.x == 0)
            for (int i = 0; i < nw; ++i) r += sh[i];
        __syncthreads();
        return r;  // valid in thread 0
    }
};
template <> struct Red<DFArith> {
    __device__ static df sum(df v, double *sh) {
        for (int o = 16; o > 0; o >>= 1) {
            df u = {__shfl_down_sync(0xffffffffu, v.hi, o), __shfl_down_sync(0xffffffffu, v.lo, o)};
            v = df_add(v, u);
        }
        const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
        float2 *s2 = reinterpret_cast<float2 *>(sh);
        if (lane == 0) s2[wid] = make_float2(v.hi, v.lo);
        __syncthreads();
        df r = df_make(0.f);
        if (threadIdx.x == 0)
            for (int i = 0; i < nw; ++i) r = df_add(r, df{s2[i].x, s2[i].y});
        __syncthreads();
        return r;
    }
};

__device__ __forceinline__ float block_max(float v, float *sh) {
    for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_down_sync(0xffffffffu, v, o));
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    if (lane == 0) sh[wid] = v;
    __syncthreads();
    float r = 0.f;
    if (threadIdx.x == 0)
        for (int i = 0; i < nw; ++i) r = fmaxf(r, sh[i]);
    __syncthreads();
    return r;
}

__device__ __forceinline__ void atomic_max_nonneg(unsigned long long *p, double v) {
    // non-negative doubles (and NaN, whose pattern is larger) order like their bit patterns
    atomicMax(p, (unsigned long long)__double_as_longlong(v));
}

// ---------------------------------------------------------------- warp helpers
template <class V> __device__ __forceinline__ V shdown(V v, int d);
template <> __device__ __forceinline__ df shdown<df>(df v, int d) {
    return {__shfl_down_sync(0xffffffffu, v.hi, d), __shfl_down_sync(0xffffffffu, v.lo, d)};
}
template <> __device__ __forceinline__ double shdown<double>(double v, int d) {
    return __shfl_down_sync(0xffffffffu, v, d);
}
template <class V> __device__ __forceinline__ V shup(V v, int d);
template <> __device__ __forceinline__ df shup<df>(df v, int d) {
    return {__shfl_up_sync(0xffffffffu, v.hi, d), __shfl_up_sync(0xffffffffu, v.lo, d)};
}
template <> __device__ __forceinline__ double shup<double>(double v, int d) { return __shfl_up_sync(0xffffffffu, v, d); }

// phi of the solve being refined: float-float (hi, lo) arrays on the mixed path
// (lo absent before the first accumulation), fp64 array on the fp64 path.
template <class A> struct PhiSrc;
template <> struct PhiSrc<DFArith> {
    const float *hi, *lo;
    __device__ __forceinline__ df get(ptrdiff_t o) const { return {__ldg(hi + o), lo ? __ldg(lo + o) : 0.f}; }
};
template <> struct PhiSrc<F64Arith> {
    const double *p;
    __device__ __forceinline__ double get(ptrdiff_t o) const { return __ldg(p + o); }
};

// Cells of a CTA's (plane, rows) block are visited by warps in 32-wide row
// segments: lanes hold consecutive i (x-neighbours by shuffle), and each warp
// walks its rows upward (y-neighbours carried in registers).  With fewer segments
// than warps the rows are split into chunks.
struct SegMap {
    int seg0, segstep, nseg, r0, r1;
};
__device__ __forceinline__ SegMap seg_map(int nx, int rows) {
    const int warp = threadIdx.x >> 5, NW = blockDim.x >> 5;
    SegMap m;
    m.nseg = (nx + 31) >> 5;
    if (m.nseg >= NW) {
        m.seg0 = warp; m.segstep = NW; m.r0 = 0; m.r1 = rows;
    } else {
        const int nchunk = NW / m.nseg;
        const int chunk = warp / m.nseg;
        m.seg0 = warp - chunk * m.nseg;
        m.segstep = m.nseg;
        if (chunk >= nchunk) {
            m.seg0 = m.nseg; m.r0 = 0; m.r1 = 0;
        } else {
            const int rpc = (rows + nchunk - 1) / nchunk;
            m.r0 = min(rows, chunk * rpc);
            m.r1 = min(rows, m.r0 + rpc);
        }
    }
    return m;
}


// one-dimensional launch grid
static inline dim3 grid1(int n) { return dim3((unsigned)n); }

}  // namespace ibf

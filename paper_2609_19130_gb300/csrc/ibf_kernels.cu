// ibf_kernels.cu -- sm_103a kernels of the pressure projection.
//
// Data flow of one solve S^-1 (Section "Fluid domain", projection paragraph: 2-D
// real FFT per x-y plane, one tridiagonal system along z per horizontal mode,
// inverse FFT), without the paper's slab transposes: the whole grid is on one GPU.
//
//   k_xfwd   per (grid, plane k, block of rows): right-hand side (divergence of u*
//            for Eq. elliptic, or the refinement residual, or the adjoint source),
//            plane sums for the singular mode, real FFT along x of two rows at a
//            time (one complex FFT of row_a + i row_b, split by symmetry), store the
//            x-spectrum in column blocks of `mb` x-modes.
//   k_yzfwd  per (grid, column block), sweeping k = 0..nz-1: FFT along y of the
//            block's columns, Thomas forward elimination for every (m, n) mode with
//            pivots from a per-plan table; overwrites the spectrum with d'_k.
//   k_00     per grid, fp64: compatibility (weighted-mean) correction, pinned solve
//            and weighted-mean normalisation of the (0,0) mode (Section "Fluid
//            Mechanics", boundary-condition paragraph: reference value of phi).
//   k_yzbwd  per (grid, column block), sweeping k = nz-1..0: back substitution,
//            inverse FFT along y.
//   k_xinv   per (grid, plane, rows): inverse real FFT along x; store phi or add
//            the refinement correction to it.
//   k_correct per cell: u = u* - alpha dt G phi (Eq. velsolen), or the adjoint output.
//
// Two precisions: fp64 (T = double, F64Arith) and mixed (T = float transforms and
// sweeps, DFArith float-float stencils / residual / accumulation, fp64 I/O converted
// with integer bit operations).
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

template <class A> struct IsDF { static constexpr bool value = false; };
template <> struct IsDF<DFArith> { static constexpr bool value = true; };

template <class A> struct Coef;
template <> struct Coef<F64Arith> {
    __device__ __forceinline__ static double c(double x) { return x; }
    __device__ __forceinline__ static double c2(float2 v, double x) { return x; }
};
template <> struct Coef<DFArith> {
    __device__ __forceinline__ static df c(double x) { return f64_to_df(x); }
    __device__ __forceinline__ static df c2(float2 v, double) { return {v.x, v.y}; }
};

template <class A> __device__ __forceinline__ float absv(typename A::V v);
template <> __device__ __forceinline__ float absv<F64Arith>(double v) { return fabsf((float)v); }
template <> __device__ __forceinline__ float absv<DFArith>(df v) { return fabsf(v.hi); }

template <typename T, class A> __device__ __forceinline__ T to_T(typename A::V v);
template <> __device__ __forceinline__ double to_T<double, F64Arith>(double v) { return v; }
template <> __device__ __forceinline__ float to_T<float, DFArith>(df v) { return df_to_f(v); }

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

// ================================================================ k_xfwd
constexpr int kRowGroup = 4;  // rows whose loads are issued together (memory-level parallelism)

// Right-hand side of one solve for a block of rows of plane k, then the real FFT
// along x of the rows (two rows per complex transform), stored as x-modes.
template <typename T, class A, int MODE>
__global__ void __launch_bounds__(kXThreads, sizeof(T) == 4 ? 2 : 1)
    k_xfwd(Work w, UserPtrs p, int use_ws, int lo_valid, double s, double rs) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    cx<T> *buf = reinterpret_cast<cx<T> *>(smem_raw);
    __shared__ double red[kXThreads / 32];
    __shared__ float redf[kXThreads / 32];
    typedef typename A::V V;

    const int b = blockIdx.x + p.blk0;
    const int g = find_grid(w.xblk_start, w.ngrids, b);
    const GridDev &G = w.grids[g];
    const int lb = b - __ldg(w.xblk_start + g);
    const int nrb = G.nrb, rows = G.rows;
    const int k = lb / nrb, rb = lb - k * nrb;
    const int j0 = rb * rows;
    const int nx = G.nx, ny = G.ny, nz = G.nz;
    const int N1 = G.nx1, N2 = G.nx2, sstride = fft_seq_len(N1, N2);
    const FDiv fN1 = G.fnx1, fN2 = G.fnx2;
    const int gi = g - p.g0;
    const int zo = G.z_off;
    const ptrdiff_t plane = (ptrdiff_t)nx * ny;
    const ptrdiff_t pbase = (ptrdiff_t)k * plane;

    V cu, cv, cwp, cwm, cp;
    if (MODE == XM_DIV) {
        const double rhz = w.z.rhz[zo + k];
        cu = Coef<A>::c(rs * G.rdx);
        cv = Coef<A>::c(rs * G.rdy);
        cwp = Coef<A>::c(rs * rhz);
        cwm = cwp;
        cp = A::zero();
    } else if (MODE == XM_ADJ) {
        const double rhz = w.z.rhz[zo + k];
        cu = Coef<A>::c(rhz * G.rdx);
        cv = Coef<A>::c(rhz * G.rdy);
        cwp = Coef<A>::c(rhz * w.z.rgzf[zo + k + 1]);
        cwm = Coef<A>::c(rhz * w.z.rgzf[zo + k]);
        cp = Coef<A>::c(rs * rhz);
    } else {  // residual b - <b> - L phi, L phi = rdx^2 d2x + rdy^2 d2y + rhz (rgzf+ dz+ - rgzf- dz-)
        cu = Coef<A>::c(G.rdx * G.rdx);
        cv = Coef<A>::c(G.rdy * G.rdy);
        const double rhz = w.z.rhz[zo + k];
        cwp = Coef<A>::c(rhz * w.z.rgzf[zo + k + 1]);
        cwm = Coef<A>::c(rhz * w.z.rgzf[zo + k]);
        cp = Coef<A>::c(w.mean_b[g]);
    }
    const T scale = (T)G.inv_nxy;

    V acc = A::zero();
    V acc_phi = A::zero();  // residual mode: plane sum of the current phi
    float vmax = 0.f;
    const int lane = threadIdx.x & 31;
    const SegMap sm = seg_map(nx, rows);
    for (int seg = sm.seg0; seg < sm.nseg; seg += sm.segstep) {
        const int i = seg * 32 + lane;
        const bool act = i < nx;
        const int ii = act ? i : nx - 1;  // inactive lanes load a valid cell and discard it
        const int ip = (ii + 1 == nx) ? 0 : ii + 1;
        const int im = (ii == 0) ? nx - 1 : ii - 1;
        const bool own_up = (lane == 31) || (ii + 1 == nx);
        const bool own_dn = (lane == 0) || (ii == 0);
        const int spos = pos_nat(ii, fN2);
        if (MODE == XM_DIV || MODE == XM_ADJ) {
            const double *u = p.in_u[gi] + pbase, *vv = p.in_v[gi] + pbase, *ww = p.in_w[gi] + pbase;
            const double *pp = (MODE == XM_ADJ && p.in_p[gi]) ? p.in_p[gi] + pbase : nullptr;
            V vcur = A::zero();
            bool have_v = false;
            for (int jg = sm.r0; jg < sm.r1; jg += kRowGroup) {
                // load phase: every fp64 input of up to kRowGroup rows is requested first
                double ru[kRowGroup], rue[kRowGroup], rvn[kRowGroup], rw0[kRowGroup], rw1[kRowGroup],
                    rp[kRowGroup];
                double rv0 = 0.0;
                const bool need_v0 = !have_v;
#pragma unroll
                for (int q = 0; q < kRowGroup; ++q) {
                    const int jl = jg + q, j = j0 + jl;
                    ru[q] = rue[q] = rvn[q] = rw0[q] = rw1[q] = rp[q] = 0.0;
                    if (jl < sm.r1 && j < ny) {
                        const int jp = (j + 1 == ny) ? 0 : j + 1;
                        const int row = j * nx;
                        ru[q] = __ldg(u + row + ii);
                        if (own_up) rue[q] = __ldg(u + row + ip);
                        if (q == 0 && need_v0) rv0 = __ldg(vv + row + ii);
                        rvn[q] = __ldg(vv + jp * nx + ii);
                        rw0[q] = __ldg(ww + row + ii);
                        rw1[q] = __ldg(ww + plane + row + ii);
                        if (MODE == XM_ADJ && pp) rp[q] = __ldg(pp + row + ii);
                    }
                }
                if (need_v0) vcur = A::load(rv0);
#pragma unroll
                for (int q = 0; q < kRowGroup; ++q) {
                    const int jl = jg + q, j = j0 + jl;
                    if (jl >= sm.r1) break;  // warp-uniform
                    T val = (T)0;
                    if (j < ny) {
                        const int row = j * nx;
                        const V U = A::load(ru[q]);
                        V Un = shdown(U, 1);
                        if (own_up) Un = A::load(rue[q]);
                        const V Vn = A::load(rvn[q]);
                        const V W0 = A::load(rw0[q]), W1 = A::load(rw1[q]);
                        V bv = A::add(A::mul(cu, A::sub(Un, U)), A::mul(cv, A::sub(Vn, vcur)));
                        if (MODE == XM_DIV) {
                            bv = A::add(bv, A::mul(cwp, A::sub(W1, W0)));
                        } else {
                            bv = A::add(bv, A::sub(A::mul(cwp, W1), A::mul(cwm, W0)));
                            if (pp) bv = A::add(bv, A::mul(cp, A::load(rp[q])));
                        }
                        vcur = Vn;
                        have_v = true;
                        if (act) {
                            if (MODE == XM_DIV) vmax = fmaxf(vmax, absv<A>(bv));
                            if (sizeof(T) == 4)
                                w.bdf[G.cell_off + pbase + row + i] = *reinterpret_cast<const float2 *>(&bv);
                            acc = A::add(acc, bv);
                            val = to_T<T, A>(bv) * scale;
                        }
                    } else {
                        have_v = false;
                    }
                    if (act) *(reinterpret_cast<T *>(buf + (jl >> 1) * sstride + spos) + (jl & 1)) = val;
                }
            }
        } else {
            PhiSrc<A> ph;
            if constexpr (sizeof(T) == 4) {
                ph.hi = w.phi_hi + G.cell_off + pbase;
                ph.lo = lo_valid ? w.phi_lo + G.cell_off + pbase : nullptr;
            }
            const float2 *bd = w.bdf + G.cell_off + pbase;
            V Pm = A::zero(), Pc = A::zero();
            bool have = false;
            for (int jg = sm.r0; jg < sm.r1; jg += kRowGroup) {
                V pn[kRowGroup], pkp[kRowGroup], pkm[kRowGroup], peu[kRowGroup], ped[kRowGroup];
                float2 bdv[kRowGroup];
                V pm0 = A::zero(), pc0 = A::zero();
                const bool need0 = !have;
#pragma unroll
                for (int q = 0; q < kRowGroup; ++q) {
                    const int jl = jg + q, j = j0 + jl;
                    pn[q] = pkp[q] = pkm[q] = peu[q] = ped[q] = A::zero();
                    bdv[q] = make_float2(0.f, 0.f);
                    if (jl < sm.r1 && j < ny) {
                        const int jp = (j + 1 == ny) ? 0 : j + 1;
                        const int jm = (j == 0) ? ny - 1 : j - 1;
                        const int row = j * nx;
                        if (q == 0 && need0) {
                            pm0 = ph.get(jm * nx + ii);
                            pc0 = ph.get(row + ii);
                        }
                        pn[q] = ph.get(jp * nx + ii);
                        if (k + 1 < nz) pkp[q] = ph.get(plane + row + ii);
                        if (k > 0) pkm[q] = ph.get(row + ii - plane);
                        if (own_up) peu[q] = ph.get(row + ip);
                        if (own_dn) ped[q] = ph.get(row + im);
                        if (act) bdv[q] = __ldg(bd + row + i);
                    }
                }
                if (need0) {
                    Pm = pm0;
                    Pc = pc0;
                }
#pragma unroll
                for (int q = 0; q < kRowGroup; ++q) {
                    const int jl = jg + q, j = j0 + jl;
                    if (jl >= sm.r1) break;
                    T val = (T)0;
                    if (j < ny) {
                        V Pip = shdown(Pc, 1);
                        if (own_up) Pip = peu[q];
                        V Pim = shup(Pc, 1);
                        if (own_dn) Pim = ped[q];
                        const V dzp = (k + 1 < nz) ? A::sub(pkp[q], Pc) : A::zero();
                        const V dzm = (k > 0) ? A::sub(Pc, pkm[q]) : A::zero();
                        const V dxp = A::sub(Pip, Pc), dxm = A::sub(Pc, Pim);
                        const V dyp = A::sub(pn[q], Pc), dym = A::sub(Pc, Pm);
                        V lap = A::add(A::mul(cu, A::sub(dxp, dxm)), A::mul(cv, A::sub(dyp, dym)));
                        lap = A::add(lap, A::sub(A::mul(cwp, dzp), A::mul(cwm, dzm)));
                        if (act) {
                            V bvv = A::zero();
                            if constexpr (sizeof(T) == 4) bvv = df{bdv[q].x, bdv[q].y};
                            const V bv = A::sub(A::sub(bvv, cp), lap);
                            acc = A::add(acc, bv);
                            acc_phi = A::add(acc_phi, Pc);
                            val = to_T<T, A>(bv) * scale;
                        }
                        Pm = Pc;
                        Pc = pn[q];
                        have = true;
                    } else {
                        have = false;
                    }
                    if (act) *(reinterpret_cast<T *>(buf + (jl >> 1) * sstride + spos) + (jl & 1)) = val;
                }
            }
        }
    }
    // plane sums of this block's rows (for the singular mode), fixed reduction order
    V tot = Red<A>::sum(acc, red);
    if (threadIdx.x == 0) w.partial[G.part_off + k * nrb + rb] = A::store(tot);
    if (MODE == XM_RESID) {
        V totp = Red<A>::sum(acc_phi, red);
        if (threadIdx.x == 0) w.partial_phi[G.part_off + k * nrb + rb] = A::store(totp);
    }
    if (MODE == XM_DIV) {
        float mx = block_max(vmax, redf);
        if (threadIdx.x == 0) atomic_max_nonneg(w.maxb + g, (double)mx);
    }
    __syncthreads();

    const cx<T> *twx = reinterpret_cast<const cx<T> *>(w.twx) + G.twx_off;
    fft_batch<T, -1>(buf, rows >> 1, sstride, N1, N2, fN1, fN2, twx);

    // split the two real rows and store x-modes m = 0..nx/2 in column blocks
    const int mb = G.mb, ncb = G.ncb, nxh = G.nxh;
    cx<T> *spec = reinterpret_cast<cx<T> *>(w.spec) + G.spec_off + (size_t)k * ncb * ny * mb;
    const int nout = ncb * rows * mb;
    const FDiv fmb = G.fmb, frows = G.frows;
    for (int t = threadIdx.x; t < nout; t += blockDim.x) {
        const int rest = (int)fdiv((unsigned)t, fmb);
        const int mm = t - rest * mb;
        const int cb = (int)fdiv((unsigned)rest, frows);
        const int jl = rest - cb * rows;
        const int m = cb * mb + mm, j = j0 + jl;
        if (m >= nxh || j >= ny) continue;
        const cx<T> *seq = buf + (jl >> 1) * sstride;
        const cx<T> Zm = seq[pos_tr(m, N1, N2, fN1)];
        const cx<T> Zc = seq[pos_tr(m == 0 ? 0 : nx - m, N1, N2, fN1)];
        cx<T> X;
        if ((jl & 1) == 0) X = {(Zm.x + Zc.x) * (T)0.5, (Zm.y - Zc.y) * (T)0.5};
        else X = {(Zm.y + Zc.y) * (T)0.5, (Zc.x - Zm.x) * (T)0.5};
        spec[((size_t)cb * ny + j) * mb + mm] = X;
    }
}

// ================================================================ k_yzfwd / k_yzbwd
template <typename T> __device__ __forceinline__ const T *zarr(const double *d, const float *f);
template <> __device__ __forceinline__ const double *zarr<double>(const double *d, const float *) { return d; }
template <> __device__ __forceinline__ const float *zarr<float>(const double *, const float *f) { return f; }

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

// y-FFT + Thomas forward elimination of one column block, sweeping k = 0..nz-1.
// Shared memory: kYZStages x [FFT buffer (mb padded sequences) | pivot chunk], then the
// Thomas state d'_{k-1} of every mode of the block.  Plane k+1 (spectrum and pivots)
// is copied with cp.async while plane k is transformed and eliminated.
template <typename T>
__global__ void __launch_bounds__(kYZThreads) k_yzfwd(Work w) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int g = find_grid(w.yzblk_start, w.ngrids, blockIdx.x);
    const GridDev &G = w.grids[g];
    const int cb = blockIdx.x - __ldg(w.yzblk_start + g);
    const int ny = G.ny, nz = G.nz, mb = G.mb, ncb = G.ncb, nxh = G.nxh;
    const int N1 = G.ny1, N2 = G.ny2, sstride = fft_seq_len(N1, N2) + 1;
    const FDiv fN1 = G.fny1, fN2 = G.fny2, fmb = G.fmb;
    const int nslot = ny * mb;
    const int nvalid = min(mb, nxh - cb * mb);  // valid x-modes of this block
    const cx<T> *twy = reinterpret_cast<const cx<T> *>(w.twy) + G.twy_off;
    const T *az = zarr<T>(w.z.az, w.z.azf) + G.z_off;
    const int tid = threadIdx.x, nthr = blockDim.x;
    const size_t fftsz = (size_t)mb * sstride;  // complex elements of one FFT buffer
    const size_t stage_bytes = ((fftsz * sizeof(cx<T>) + (size_t)nslot * sizeof(T)) + 15) & ~(size_t)15;
    auto fbuf = [&](int st) { return reinterpret_cast<cx<T> *>(smem_raw + st * stage_bytes); };
    auto tbuf = [&](int st) { return reinterpret_cast<T *>(smem_raw + st * stage_bytes + fftsz * sizeof(cx<T>)); };
    cx<T> *state = reinterpret_cast<cx<T> *>(smem_raw + kYZStages * stage_bytes);
    const cx<T> *spec = reinterpret_cast<const cx<T> *>(w.spec) + G.spec_off;
    cx<T> *specw = reinterpret_cast<cx<T> *>(w.spec) + G.spec_off;
    const T *tab = reinterpret_cast<const T *>(w.tab) + G.tab_off;

    auto issue = [&](int k) {
        if (k < nz) {
            const int st = k % kYZStages;
            cx<T> *fb = fbuf(st);
            T *tb = tbuf(st);
            const cx<T> *src = spec + ((size_t)k * ncb + cb) * nslot;
            const T *tsrc = tab + ((size_t)k * ncb + cb) * nslot;
            for (int t = tid; t < nslot; t += nthr) {
                const int j = (int)fdiv((unsigned)t, fmb), mm = t - j * mb;
                cx<T> *dst = fb + mm * sstride + pos_nat(j, fN2);
                if (mm < nvalid) cp_async<sizeof(cx<T>)>(dst, src + t);
                else *dst = {(T)0, (T)0};
                cp_async<sizeof(T)>(tb + t, tsrc + t);
            }
        }
        cp_async_commit();
    };

    for (int q = tid; q < nslot; q += nthr) state[q] = {(T)0, (T)0};
    for (int k = 0; k < kYZStages - 1; ++k) issue(k);

    for (int k = 0; k < nz; ++k) {
        issue(k + kYZStages - 1);
        cp_async_wait<kYZStages - 1>();
        __syncthreads();
        cx<T> *buf = fbuf(k % kYZStages);
        const T *tb = tbuf(k % kYZStages);
        fft_batch<T, -1>(buf, mb, sstride, N1, N2, fN1, fN2, twy);
        cx<T> *pl = specw + ((size_t)k * ncb + cb) * nslot;
        const T a = az[k];
        for (int q = tid; q < nslot; q += nthr) {
            const int sn = (int)fdiv((unsigned)q, fmb), mm = q - sn * mb;
            const cx<T> rin = buf[mm * sstride + pos_nat(sn, fN2)];
            const T inv = tb[q];
            const cx<T> dp = state[q];
            cx<T> d = {(rin.x - a * dp.x) * inv, (rin.y - a * dp.y) * inv};
            if (cb == 0 && q == 0) d = rin;  // (0,0) mode: solved by k_00
            state[q] = d;
            if (mm < nvalid) pl[q] = d;
        }
        __syncthreads();
    }
    cp_async_wait<0>();
}

// Back substitution and inverse y-FFT of one column block, sweeping k = nz-1..0.
// Shared memory: kYZStages x [d' chunk (slot order) | pivot chunk], then one FFT
// buffer and the state phi_hat_{k+1}; plane k-1 is copied while plane k is processed.
template <typename T>
__global__ void __launch_bounds__(kYZThreads) k_yzbwd(Work w) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int g = find_grid(w.yzblk_start, w.ngrids, blockIdx.x);
    const GridDev &G = w.grids[g];
    const int cb = blockIdx.x - __ldg(w.yzblk_start + g);
    const int ny = G.ny, nz = G.nz, mb = G.mb, ncb = G.ncb, nxh = G.nxh;
    const int N1 = G.ny1, N2 = G.ny2, sstride = fft_seq_len(N1, N2) + 1;
    const FDiv fN1 = G.fny1, fN2 = G.fny2, fmb = G.fmb;
    const int nslot = ny * mb;
    const int nvalid = min(mb, nxh - cb * mb);
    const cx<T> *twy = reinterpret_cast<const cx<T> *>(w.twy) + G.twy_off;
    const T *cz = zarr<T>(w.z.cz, w.z.czf) + G.z_off;
    const int tid = threadIdx.x, nthr = blockDim.x;
    const size_t stage_bytes = (((size_t)nslot * (sizeof(cx<T>) + sizeof(T))) + 15) & ~(size_t)15;
    auto dbuf = [&](int st) { return reinterpret_cast<cx<T> *>(smem_raw + st * stage_bytes); };
    auto tbuf = [&](int st) { return reinterpret_cast<T *>(smem_raw + st * stage_bytes + (size_t)nslot * sizeof(cx<T>)); };
    cx<T> *buf = reinterpret_cast<cx<T> *>(smem_raw + kYZStages * stage_bytes);
    cx<T> *state = buf + (size_t)mb * sstride;
    cx<T> *spec = reinterpret_cast<cx<T> *>(w.spec) + G.spec_off;
    const T *tab = reinterpret_cast<const T *>(w.tab) + G.tab_off;

    auto issue = [&](int k) {  // plane k (k >= 0) into stage (nz-1-k) % S
        if (k >= 0) {
            const int st = (nz - 1 - k) % kYZStages;
            cx<T> *db = dbuf(st);
            T *tb = tbuf(st);
            const cx<T> *src = spec + ((size_t)k * ncb + cb) * nslot;
            const T *tsrc = tab + ((size_t)k * ncb + cb) * nslot;
            for (int t = tid; t < nslot; t += nthr) {
                const int sn = (int)fdiv((unsigned)t, fmb), mm = t - sn * mb;
                if (mm < nvalid) cp_async<sizeof(cx<T>)>(db + t, src + t);
                else db[t] = {(T)0, (T)0};
                cp_async<sizeof(T)>(tb + t, tsrc + t);
            }
        }
        cp_async_commit();
    };

    for (int q = tid; q < nslot; q += nthr) state[q] = {(T)0, (T)0};
    for (int s_ = 0; s_ < kYZStages - 1; ++s_) issue(nz - 1 - s_);

    for (int k = nz - 1; k >= 0; --k) {
        issue(k - (kYZStages - 1));
        cp_async_wait<kYZStages - 1>();
        __syncthreads();
        const int st = (nz - 1 - k) % kYZStages;
        const cx<T> *db = dbuf(st);
        const T *tb = tbuf(st);
        const T c = cz[k];
        for (int q = tid; q < nslot; q += nthr) {
            const int sn = (int)fdiv((unsigned)q, fmb), mm = q - sn * mb;
            const cx<T> d = db[q];
            const T cp = c * tb[q];
            const cx<T> nx_ = state[q];
            cx<T> ph = {d.x - cp * nx_.x, d.y - cp * nx_.y};
            if (cb == 0 && q == 0) ph = d;
            state[q] = ph;
            buf[mm * sstride + pos_nat(sn, fN2)] = ph;
        }
        __syncthreads();
        fft_batch<T, +1>(buf, mb, sstride, N1, N2, fN1, fN2, twy);
        cx<T> *pl = spec + ((size_t)k * ncb + cb) * nslot;
        for (int t = tid; t < nslot; t += nthr) {
            const int j = (int)fdiv((unsigned)t, fmb), mm = t - j * mb;
            if (mm < nvalid) pl[t] = buf[mm * sstride + pos_nat(j, fN2)];
        }
        __syncthreads();
    }
    cp_async_wait<0>();
}

// ================================================================ k_00 (fp64, one CTA per grid)
template <typename T>
__global__ void __launch_bounds__(256) k_00(Work w, int first_solve) {
    // Shared memory: right-hand side, hz, and two copies (ping-pong) of the four PCR
    // arrays a, b, c, d; every array has nz+1 entries.
    extern __shared__ double sh00[];
    __shared__ double red[8];
    const int g = blockIdx.x;
    const GridDev &G = w.grids[g];
    const int nz = G.nz, nrb = G.nrb, zo = G.z_off;
    const int L = nz + 1;
    double *rhs = sh00, *hz = sh00 + L;
    double *A0 = sh00 + 2 * L, *B0 = A0 + L, *C0 = B0 + L, *D0 = C0 + L;
    double *A1 = D0 + L, *B1 = A1 + L, *C1 = B1 + L, *D1 = C1 + L;
    const double *part = w.partial + G.part_off;
    double loc = 0.0, locp = 0.0;
    bool bad = false;
    for (int k = threadIdx.x; k < nz; k += blockDim.x) {
        double S = 0.0;
        for (int r = 0; r < nrb; ++r) S += part[k * nrb + r];
        const double m = S * G.inv_nxy;  // plane mean of the right-hand side
        if (!isfinite(m)) bad = true;
        const double h = w.z.hz[zo + k];
        rhs[k] = m;
        hz[k] = h;
        loc += h * m;
        if (!first_solve) {
            double P = 0.0;
            for (int r = 0; r < nrb; ++r) P += w.partial_phi[G.part_off + k * nrb + r];
            locp += h * P * G.inv_nxy;
        }
    }
    if (bad) atomicOr(w.err, 1u << 6);  // IBF_ERR_NONFINITE
    __syncthreads();
    const double tot = Red<F64Arith>::sum(loc, red);
    // weighted mean of the phi being refined: the correction also removes it, so that
    // phi + delta keeps a zero weighted mean (L cannot see a constant)
    const double totp = first_solve ? 0.0 : Red<F64Arith>::sum(locp, red);
    if (threadIdx.x == 0) red[0] = tot / G.sum_hz;
    __syncthreads();
    const double mean = red[0];
    if (threadIdx.x == 0 && first_solve) {
        w.mean_b[g] = mean;
        double scale = 0.0;
        for (int k = 0; k < nz; ++k) scale = fmax(scale, fabs(rhs[k]));
        // compatibility defect large compared with the plane means -> warning
        if (fabs(mean) > 1e-8 * scale && fabs(mean) > 0.0) atomicOr(w.err, 1u << 7);
    }
    // Pinned system (level 0 fixed to zero, so row 0 reads phi_0 = 0) solved by
    // parallel cyclic reduction (Hockney 1965): each step eliminates from every row its
    // couplings at distance st; after ceil(log2 nz) steps row k reads phi_k = d_k / b_k.
    // Row k of L along z: a = az_k (to k-1), b = -(az_k + cz_k), c = cz_k (to k+1).
    for (int k = threadIdx.x; k < nz; k += blockDim.x) {
        if (k == 0) { A0[k] = 0.0; B0[k] = 1.0; C0[k] = 0.0; D0[k] = 0.0; }
        else {
            const double a = w.z.az[zo + k], c = w.z.cz[zo + k];
            A0[k] = a; B0[k] = -(a + c); C0[k] = (k == 0) ? 0.0 : c; D0[k] = rhs[k] - mean;
        }
    }
    __syncthreads();
    for (int st = 1; st < nz; st <<= 1) {
        for (int k = threadIdx.x; k < nz; k += blockDim.x) {
            double na = 0.0, nb = B0[k], nc = 0.0, nd = D0[k];
            if (k - st >= 0) {
                const double al = -A0[k] / B0[k - st];
                na = al * A0[k - st];
                nb += al * C0[k - st];
                nd += al * D0[k - st];
            }
            if (k + st < nz) {
                const double ga = -C0[k] / B0[k + st];
                nc = ga * C0[k + st];
                nb += ga * A0[k + st];
                nd += ga * D0[k + st];
            }
            A1[k] = na; B1[k] = nb; C1[k] = nc; D1[k] = nd;
        }
        __syncthreads();
        double *t;
        t = A0; A0 = A1; A1 = t;
        t = B0; B0 = B1; B1 = t;
        t = C0; C0 = C1; C1 = t;
        t = D0; D0 = D1; D1 = t;
    }
    double lsv = 0.0;
    for (int k = threadIdx.x; k < nz; k += blockDim.x) {
        const double ph = D0[k] / B0[k];
        rhs[k] = ph;
        lsv += hz[k] * ph;
    }
    __syncthreads();
    const double sv = Red<F64Arith>::sum(lsv, red);
    if (threadIdx.x == 0) rhs[nz] = (sv + totp) / G.sum_hz;  // weighted mean to remove
    __syncthreads();
    const double mphi = rhs[nz];
    cx<T> *spec = reinterpret_cast<cx<T> *>(w.spec) + G.spec_off;
    const size_t stride = (size_t)G.ncb * G.ny * G.mb;
    for (int k = threadIdx.x; k < nz; k += blockDim.x) spec[(size_t)k * stride] = {(T)(rhs[k] - mphi), (T)0};
}

// ================================================================ k_xinv
// Inverse real FFT along x of a block of rows; STORE writes phi (fp64 path: fp64
// array; mixed path: the hi array of the float-float phi), ACCUM adds the
// refinement correction to the float-float phi.
template <typename T, class A, int IMODE>
__global__ void __launch_bounds__(kXThreads, sizeof(T) == 4 ? 2 : 1)
    k_xinv(Work w, UserPtrs p, int use_ws, int lo_valid) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    cx<T> *buf = reinterpret_cast<cx<T> *>(smem_raw);
    const int b = blockIdx.x + p.blk0;
    const int g = find_grid(w.xblk_start, w.ngrids, b);
    const GridDev &G = w.grids[g];
    const int lb = b - __ldg(w.xblk_start + g);
    const int nrb = G.nrb, rows = G.rows;
    const int k = lb / nrb, rb = lb - k * nrb;
    const int j0 = rb * rows;
    const int nx = G.nx, ny = G.ny;
    const int N1 = G.nx1, N2 = G.nx2, sstride = fft_seq_len(N1, N2);
    const FDiv fN1 = G.fnx1, fN2 = G.fnx2, fmb = G.fmb, fnpair = G.fnpair, fnx = G.fnx;
    const int mb = G.mb, ncb = G.ncb, nxh = G.nxh;
    const cx<T> *spec = reinterpret_cast<const cx<T> *>(w.spec) + G.spec_off + (size_t)k * ncb * ny * mb;
    const int npair = rows >> 1;
    const int nload = ncb * npair * mb;
    for (int t = threadIdx.x; t < nload; t += blockDim.x) {
        const int rest = (int)fdiv((unsigned)t, fmb);
        const int mm = t - rest * mb;
        const int cb = (int)fdiv((unsigned)rest, fnpair);
        const int s_ = rest - cb * npair;
        const int m = cb * mb + mm;
        if (m >= nxh) continue;
        const int ja = j0 + 2 * s_, jb = ja + 1;
        cx<T> A_ = {(T)0, (T)0}, B_ = {(T)0, (T)0};
        if (ja < ny) A_ = spec[((size_t)cb * ny + ja) * mb + mm];
        if (jb < ny) B_ = spec[((size_t)cb * ny + jb) * mb + mm];
        cx<T> *seq = buf + s_ * sstride;
        seq[pos_tr(m, N1, N2, fN1)] = {A_.x - B_.y, A_.y + B_.x};
        if (m > 0 && 2 * m < nx) seq[pos_tr(nx - m, N1, N2, fN1)] = {A_.x + B_.y, B_.x - A_.y};
    }
    __syncthreads();
    const cx<T> *twx = reinterpret_cast<const cx<T> *>(w.twx) + G.twx_off;
    fft_batch<T, +1>(buf, npair, sstride, N1, N2, fN1, fN2, twx);

    const int gi = g - p.g0;
    const ptrdiff_t plane = (ptrdiff_t)nx * ny;
    const ptrdiff_t base = (ptrdiff_t)k * plane + (ptrdiff_t)j0 * nx;
    const int ncell = min(rows, ny - j0) * nx;
    double *phi64 = nullptr;
    float *phh = nullptr, *phl = nullptr;
    if (sizeof(T) == 8) phi64 = (use_ws ? (w.phi_ws + G.cell_off) : p.out_p[gi]) + base;
    else {
        phh = w.phi_hi + G.cell_off + base;
        phl = w.phi_lo + G.cell_off + base;
    }
    for (int t = threadIdx.x; t < ncell; t += blockDim.x) {
        const int jl = (int)fdiv((unsigned)t, fnx), i = t - jl * nx;
        const cx<T> z = buf[(jl >> 1) * sstride + pos_nat(i, fN2)];
        const T val = (jl & 1) ? z.y : z.x;
        if constexpr (sizeof(T) == 8) {
            phi64[t] = (double)val;
        } else {
            if (IMODE == IM_STORE) {
                phh[t] = (float)val;
            } else if (!lo_valid) {
                phl[t] = (float)val;  // phi = phi_0 + delta held as the unevaluated pair (hi, lo)
            } else {
                const df cur = {phh[t], phl[t]};
                const df nw = df_addf(cur, (float)val);
                phh[t] = nw.hi;
                phl[t] = nw.lo;
            }
        }
    }
}

// ================================================================ k_correct
constexpr int kRowGroupC = 2;

// forward (ADJ = 0): u = u* + s rdx (phi_{i-1} - phi_i), v likewise,
//                    w_k = w*_k + s rgzf_k (phi_{k-1} - phi_k), wall faces copied;
//                    mixed path: also writes phi (fp64) from its float-float value.
// adjoint (ADJ = 1): g* = g_u + hz_k rdx (psi_{i-1} - psi_i), ...,
//                    w_k = g_w,k + psi_{k-1} [k>=1] - psi_k [k<=nz-1].
template <class A, int ADJ>
__global__ void __launch_bounds__(kXThreads, 4) k_correct(Work w, UserPtrs p, int use_ws, int lo_valid, double s) {
    typedef typename A::V V;
    const int b = blockIdx.x + p.blk0;
    const int g = find_grid(w.xblk_start, w.ngrids, b);
    const GridDev &G = w.grids[g];
    const int lb = b - __ldg(w.xblk_start + g);
    const int nrb = G.nrb, rows = G.rows;
    const int k = lb / nrb, rb = lb - k * nrb;
    const int j0 = rb * rows;
    const int nx = G.nx, ny = G.ny, nz = G.nz;
    const int gi = g - p.g0;
    const int zo = G.z_off;
    const ptrdiff_t plane = (ptrdiff_t)nx * ny;
    const ptrdiff_t pbase = (ptrdiff_t)k * plane;
    PhiSrc<A> ph;
    constexpr bool MIX = IsDF<A>::value;
    if constexpr (MIX) {
        ph.hi = w.phi_hi + G.cell_off + pbase;
        ph.lo = lo_valid ? w.phi_lo + G.cell_off + pbase : nullptr;
    } else {
        ph.p = (use_ws ? (w.phi_ws + G.cell_off) : p.out_p[gi]) + pbase;
    }
    const double *ui = p.in_u[gi] + pbase, *vi = p.in_v[gi] + pbase, *wi = p.in_w[gi] + pbase;
    double *uo = p.out_u[gi] + pbase, *vo = p.out_v[gi] + pbase, *wo = p.out_w[gi] + pbase;
    double *po = (MIX && !ADJ) ? p.out_p[gi] + pbase : nullptr;
    V cu, cv, cw;
    if (ADJ) {
        const double hz = w.z.hz[zo + k];
        cu = Coef<A>::c(hz * G.rdx);
        cv = Coef<A>::c(hz * G.rdy);
        cw = Coef<A>::c(1.0);
    } else {
        cu = Coef<A>::c(s * G.rdx);
        cv = Coef<A>::c(s * G.rdy);
        cw = Coef<A>::c(s * w.z.rgzf[zo + k]);
    }
    const int lane = threadIdx.x & 31;
    const SegMap sm = seg_map(nx, rows);
    for (int seg = sm.seg0; seg < sm.nseg; seg += sm.segstep) {
        const int i = seg * 32 + lane;
        const bool act = i < nx;
        const int ii = act ? i : nx - 1;
        const int im = (ii == 0) ? nx - 1 : ii - 1;
        const bool own_dn = (lane == 0) || (ii == 0);
        V Pjm = A::zero();
        bool have = false;
        for (int jg = sm.r0; jg < sm.r1; jg += kRowGroupC) {
            V pc[kRowGroupC], pkm[kRowGroupC], ped[kRowGroupC];
            double ru[kRowGroupC], rv[kRowGroupC], rw[kRowGroupC], rwt[kRowGroupC];
            V pjm0 = A::zero();
            const bool need0 = !have;
#pragma unroll
            for (int q = 0; q < kRowGroupC; ++q) {
                const int jl = jg + q, j = j0 + jl;
                pc[q] = pkm[q] = ped[q] = A::zero();
                ru[q] = rv[q] = rw[q] = rwt[q] = 0.0;
                if (jl < sm.r1 && j < ny) {
                    const int jm = (j == 0) ? ny - 1 : j - 1;
                    const int row = j * nx;
                    if (q == 0 && need0) pjm0 = ph.get(jm * nx + ii);
                    pc[q] = ph.get(row + ii);
                    if (k > 0) pkm[q] = ph.get(row + ii - plane);
                    if (own_dn) ped[q] = ph.get(row + im);
                    if (act) {
                        ru[q] = ui[row + i];
                        rv[q] = vi[row + i];
                        rw[q] = wi[row + i];
                        if (k == nz - 1) rwt[q] = wi[row + i + plane];
                    }
                }
            }
            if (need0) Pjm = pjm0;
#pragma unroll
            for (int q = 0; q < kRowGroupC; ++q) {
                const int jl = jg + q, j = j0 + jl;
                if (jl >= sm.r1 || j >= ny) break;  // warp-uniform
                const int row = j * nx;
                const V Pc = pc[q];
                V Pim = shup(Pc, 1);
                if (own_dn) Pim = ped[q];
                if (act) {
                    // the correction t is formed in the solve's high precision; the face
                    // value u* + t is one fp64 add (the fp64 pipe is otherwise idle here)
                    const int c = row + i;
                    uo[c] = ru[q] + A::store(A::mul(cu, A::sub(Pim, Pc)));
                    vo[c] = rv[q] + A::store(A::mul(cv, A::sub(Pjm, Pc)));
                    if (ADJ) {
                        wo[c] = rw[q] + A::store(A::sub(pkm[q], Pc));
                        if (k == nz - 1) wo[c + plane] = rwt[q] + A::store(A::norm(Pc));
                    } else {
                        if (k == 0) wo[c] = rw[q];
                        else wo[c] = rw[q] + A::store(A::mul(cw, A::sub(pkm[q], Pc)));
                        if (k == nz - 1) wo[c + plane] = rwt[q];
                        if (po) po[c] = A::store(A::norm(Pc));
                    }
                }
                Pjm = Pc;
                have = true;
            }
        }
    }
}

// ================================================================ k_divstat: max |D u| of the output
template <class A>
__global__ void __launch_bounds__(kXThreads) k_divstat(Work w, UserPtrs p) {
    typedef typename A::V V;
    __shared__ float redf[kXThreads / 32];
    const int b = blockIdx.x + p.blk0;
    const int g = find_grid(w.xblk_start, w.ngrids, b);
    const GridDev &G = w.grids[g];
    const int lb = b - __ldg(w.xblk_start + g);
    const int nrb = G.nrb, rows = G.rows;
    const int k = lb / nrb, rb = lb - k * nrb;
    const int j0 = rb * rows;
    const int nx = G.nx, ny = G.ny;
    const int gi = g - p.g0;
    const ptrdiff_t plane = (ptrdiff_t)nx * ny;
    const ptrdiff_t pbase = (ptrdiff_t)k * plane;
    const double *u = p.out_u[gi] + pbase, *vv = p.out_v[gi] + pbase, *ww = p.out_w[gi] + pbase;
    const V cu = Coef<A>::c(G.rdx), cv = Coef<A>::c(G.rdy), cw = Coef<A>::c(w.z.rhz[G.z_off + k]);
    float mx = 0.f;
    const int ncell = min(rows, ny - j0) * nx;
    for (int t = threadIdx.x; t < ncell; t += blockDim.x) {
        const int jl = (int)fdiv((unsigned)t, G.fnx), i = t - jl * nx;
        const int j = j0 + jl;
        const int ip = (i + 1 == nx) ? 0 : i + 1;
        const int jp = (j + 1 == ny) ? 0 : j + 1;
        const int row = j * nx;
        V d = A::mul(cu, A::sub(A::load(u[row + ip]), A::load(u[row + i])));
        d = A::add(d, A::mul(cv, A::sub(A::load(vv[jp * nx + i]), A::load(vv[row + i]))));
        d = A::add(d, A::mul(cw, A::sub(A::load(ww[plane + row + i]), A::load(ww[row + i]))));
        const float a = absv<A>(d);
        mx = (a > mx || a != a) ? a : mx;
    }
    const float r = block_max(mx, redf);
    if (threadIdx.x == 0) atomic_max_nonneg(w.maxdiv + g, (double)r);
}

// ================================================================ small kernels
__global__ void k_finalize(Work w, double *max_div, double *max_div_in, double *compat, double s) {
    const int g = blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= w.ngrids) return;
    if (max_div) max_div[g] = __longlong_as_double((long long)w.maxdiv[g]);
    if (max_div_in) max_div_in[g] = s * __longlong_as_double((long long)w.maxb[g]);
    if (compat) compat[g] = w.mean_b[g];
}

// Pivots of every mode's tridiagonal system (fp64 arithmetic, stored as T):
// inv_k = 1/(bz_k + lambda - az_k c'_{k-1}),  c'_k = cz_k inv_k,  bz_k = -(az_k + cz_k),
// lambda = -4/dx^2 sin^2(pi m/nx) - 4/dy^2 sin^2(pi n/ny).
template <typename T>
__global__ void __launch_bounds__(256) k_build_table(Work w) {
    const int g = find_grid(w.yzblk_start, w.ngrids, blockIdx.x);
    const GridDev &G = w.grids[g];
    const int cb = blockIdx.x - w.yzblk_start[g];
    const int ny = G.ny, nz = G.nz, mb = G.mb, ncb = G.ncb;
    const int N1 = G.ny1, N2 = G.ny2;
    const int nslot = ny * mb;
    const double *az = w.z.az + G.z_off, *cz = w.z.cz + G.z_off;
    T *tab = reinterpret_cast<T *>(w.tab) + G.tab_off;
    for (int q = threadIdx.x; q < nslot; q += blockDim.x) {
        const int mm = q % mb, sn = q / mb;
        const int n = (sn / N2) + N1 * (sn % N2);
        const int m = cb * mb + mm;
        const bool valid = (m < G.nxh) && !(m == 0 && n == 0);
        const double sx = sinpi((double)m / G.nx), sy = sinpi((double)n / ny);
        const double lam = -4.0 * G.rdx * G.rdx * sx * sx - 4.0 * G.rdy * G.rdy * sy * sy;
        double cp = 0.0;
        for (int k = 0; k < nz; ++k) {
            double inv = 0.0;
            if (valid) {
                inv = 1.0 / (-(az[k] + cz[k]) + lam - az[k] * cp);
                cp = cz[k] * inv;
            }
            tab[((size_t)k * ncb + cb) * nslot + q] = (T)inv;
        }
    }
}

// ================================================================ launchers
static inline dim3 grid1(int n) { return dim3((unsigned)n); }

cudaError_t launch_xfwd(int mixed, int mode, const Work &w, const UserPtrs &p, int use_ws, int lo_valid, int nblk,
                        double s, double rs, size_t smem, cudaStream_t st) {
    if (nblk <= 0) return cudaSuccess;
    if (mixed) {
        if (mode == XM_DIV)
            k_xfwd<float, DFArith, XM_DIV><<<grid1(nblk), kXThreads, smem, st>>>(w, p, use_ws, lo_valid, s, rs);
        else if (mode == XM_RESID)
            k_xfwd<float, DFArith, XM_RESID><<<grid1(nblk), kXThreads, smem, st>>>(w, p, use_ws, lo_valid, s, rs);
        else
            k_xfwd<float, DFArith, XM_ADJ><<<grid1(nblk), kXThreads, smem, st>>>(w, p, use_ws, lo_valid, s, rs);
    } else {
        if (mode == XM_DIV)
            k_xfwd<double, F64Arith, XM_DIV><<<grid1(nblk), kXThreads, smem, st>>>(w, p, use_ws, lo_valid, s, rs);
        else if (mode == XM_ADJ)
            k_xfwd<double, F64Arith, XM_ADJ><<<grid1(nblk), kXThreads, smem, st>>>(w, p, use_ws, lo_valid, s, rs);
        else
            return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

cudaError_t launch_yzfwd(int mixed, const Work &w, int nblk, size_t smem, cudaStream_t st) {
    if (mixed) k_yzfwd<float><<<grid1(nblk), kYZThreads, smem, st>>>(w);
    else k_yzfwd<double><<<grid1(nblk), kYZThreads, smem, st>>>(w);
    return cudaGetLastError();
}

cudaError_t launch_yzbwd(int mixed, const Work &w, int nblk, size_t smem, cudaStream_t st) {
    if (mixed) k_yzbwd<float><<<grid1(nblk), kYZThreads, smem, st>>>(w);
    else k_yzbwd<double><<<grid1(nblk), kYZThreads, smem, st>>>(w);
    return cudaGetLastError();
}

cudaError_t launch_k00(const Work &w, int mixed, int first_solve, int maxnz, cudaStream_t st) {
    const size_t smem = (size_t)10 * (maxnz + 1) * sizeof(double);
    if (mixed) k_00<float><<<w.ngrids, 256, smem, st>>>(w, first_solve);
    else k_00<double><<<w.ngrids, 256, smem, st>>>(w, first_solve);
    return cudaGetLastError();
}

cudaError_t launch_xinv(int mixed, int mode, const Work &w, const UserPtrs &p, int use_ws, int lo_valid, int nblk,
                        size_t smem, cudaStream_t st) {
    if (nblk <= 0) return cudaSuccess;
    if (mixed) {
        if (mode == IM_STORE)
            k_xinv<float, DFArith, IM_STORE><<<grid1(nblk), kXThreads, smem, st>>>(w, p, use_ws, lo_valid);
        else
            k_xinv<float, DFArith, IM_ACCUM><<<grid1(nblk), kXThreads, smem, st>>>(w, p, use_ws, lo_valid);
    } else {
        k_xinv<double, F64Arith, IM_STORE><<<grid1(nblk), kXThreads, smem, st>>>(w, p, use_ws, lo_valid);
    }
    return cudaGetLastError();
}

cudaError_t launch_correct(int mixed, int adjoint, const Work &w, const UserPtrs &p, int use_ws, int lo_valid,
                           int nblk, double s, cudaStream_t st) {
    if (nblk <= 0) return cudaSuccess;
    if (mixed) {
        if (adjoint) k_correct<DFArith, 1><<<grid1(nblk), kXThreads, 0, st>>>(w, p, use_ws, lo_valid, s);
        else k_correct<DFArith, 0><<<grid1(nblk), kXThreads, 0, st>>>(w, p, use_ws, lo_valid, s);
    } else {
        if (adjoint) k_correct<F64Arith, 1><<<grid1(nblk), kXThreads, 0, st>>>(w, p, use_ws, lo_valid, s);
        else k_correct<F64Arith, 0><<<grid1(nblk), kXThreads, 0, st>>>(w, p, use_ws, lo_valid, s);
    }
    return cudaGetLastError();
}

cudaError_t launch_divstat(int mixed, const Work &w, const UserPtrs &p, int nblk, cudaStream_t st) {
    if (nblk <= 0) return cudaSuccess;
    if (mixed) k_divstat<DFArith><<<grid1(nblk), kXThreads, 0, st>>>(w, p);
    else k_divstat<F64Arith><<<grid1(nblk), kXThreads, 0, st>>>(w, p);
    return cudaGetLastError();
}

cudaError_t launch_finalize(const Work &w, double *max_div, double *max_div_in, double *compat, double s,
                            cudaStream_t st) {
    k_finalize<<<(w.ngrids + 127) / 128, 128, 0, st>>>(w, max_div, max_div_in, compat, s);
    return cudaGetLastError();
}

cudaError_t launch_build_table(int mixed, const Work &w, int nblk, cudaStream_t st) {
    if (mixed) k_build_table<float><<<grid1(nblk), 256, 0, st>>>(w);
    else k_build_table<double><<<grid1(nblk), 256, 0, st>>>(w);
    return cudaGetLastError();
}

// Dynamic shared-memory caps are per-kernel attributes shared by every plan in the
// process: each is set to the device's opt-in maximum minus the kernel's static shared
// memory, so that no plan can lower them under another plan's launch size.
cudaError_t set_smem_limits(int mixed) {
    int dev = 0, optin = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    auto set = [&](const void *fn) {
        if (e != cudaSuccess) return;
        cudaFuncAttributes a;
        e = cudaFuncGetAttributes(&a, fn);
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, optin - (int)a.sharedSizeBytes);
    };
    if (mixed) {
        set((const void *)k_xfwd<float, DFArith, XM_DIV>);
        set((const void *)k_xfwd<float, DFArith, XM_RESID>);
        set((const void *)k_xfwd<float, DFArith, XM_ADJ>);
        set((const void *)k_xinv<float, DFArith, IM_STORE>);
        set((const void *)k_xinv<float, DFArith, IM_ACCUM>);
        set((const void *)k_yzfwd<float>);
        set((const void *)k_yzbwd<float>);
        set((const void *)k_00<float>);
    } else {
        set((const void *)k_xfwd<double, F64Arith, XM_DIV>);
        set((const void *)k_xfwd<double, F64Arith, XM_ADJ>);
        set((const void *)k_xinv<double, F64Arith, IM_STORE>);
        set((const void *)k_yzfwd<double>);
        set((const void *)k_yzbwd<double>);
        set((const void *)k_00<double>);
    }
    return e;
}

}  // namespace ibf

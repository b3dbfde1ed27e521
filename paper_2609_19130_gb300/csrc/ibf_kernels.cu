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

// ================================================================ k_xfwd
template <typename T, class A, int MODE>
__global__ void __launch_bounds__(kXThreads, sizeof(T) == 4 ? 2 : 1) k_xfwd(Work w, UserPtrs p, int use_ws, double s, double rs) {
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
    const int gi = g - p.g0;
    const int zo = G.z_off;
    const size_t plane = (size_t)nx * ny;

    // per-CTA coefficients
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
    } else {  // residual: b - <b> - L phi,  L phi = rdx^2 d2x + rdy^2 d2y + rhz (rgzf+ dz+ - rgzf- dz-)
        cu = Coef<A>::c(G.rdx * G.rdx);
        cv = Coef<A>::c(G.rdy * G.rdy);
        const double rhz = w.z.rhz[zo + k];
        cwp = Coef<A>::c(rhz * w.z.rgzf[zo + k + 1]);
        cwm = Coef<A>::c(rhz * w.z.rgzf[zo + k]);
        cp = Coef<A>::c(w.mean_b[g]);
    }
    const T scale = (T)G.inv_nxy;

    V acc = A::zero();
    V acc_phi = A::zero();  // residual mode: plane sum of the current phi (for its weighted mean)
    float vmax = 0.f;
    const int ncell = rows * nx;
    for (int t = threadIdx.x; t < ncell; t += blockDim.x) {
        const int jl = t / nx, i = t - jl * nx;
        const int j = j0 + jl;
        T val = (T)0;
        if (j < ny) {
            const int ip = (i + 1 == nx) ? 0 : i + 1;
            const int jp = (j + 1 == ny) ? 0 : j + 1;
            const size_t c = (size_t)k * plane + (size_t)j * nx + i;
            V bv;
            if (MODE == XM_DIV || MODE == XM_ADJ) {
                const double *u = p.in_u[gi], *vv = p.in_v[gi], *ww = p.in_w[gi];
                const size_t rowk = (size_t)k * plane + (size_t)j * nx;
                V du = A::sub(A::load(__ldg(u + rowk + ip)), A::load(__ldg(u + rowk + i)));
                V dv = A::sub(A::load(__ldg(vv + (size_t)k * plane + (size_t)jp * nx + i)), A::load(__ldg(vv + c)));
                V w1 = A::load(__ldg(ww + c + plane)), w0 = A::load(__ldg(ww + c));
                bv = A::add(A::mul(cu, du), A::mul(cv, dv));
                if (MODE == XM_DIV) bv = A::add(bv, A::mul(cwp, A::sub(w1, w0)));
                else {
                    bv = A::add(bv, A::sub(A::mul(cwp, w1), A::mul(cwm, w0)));
                    if (p.in_p[gi]) bv = A::add(bv, A::mul(cp, A::load(__ldg(p.in_p[gi] + c))));
                }
                if (MODE == XM_DIV) vmax = fmaxf(vmax, absv<A>(bv));
                if (sizeof(T) == 4) w.bdf[G.cell_off + c] = *reinterpret_cast<const float2 *>(&bv);
            } else {
                const double *ph = use_ws ? (w.phi_ws + G.cell_off) : p.out_p[gi];
                const int im = (i == 0) ? nx - 1 : i - 1;
                const int jm = (j == 0) ? ny - 1 : j - 1;
                const size_t rowk = (size_t)k * plane + (size_t)j * nx;
                const V pc = A::load(__ldg(ph + c));
                acc_phi = A::add(acc_phi, pc);
                const V dxp = A::sub(A::load(__ldg(ph + rowk + ip)), pc);
                const V dxm = A::sub(pc, A::load(__ldg(ph + rowk + im)));
                const V dyp = A::sub(A::load(__ldg(ph + (size_t)k * plane + (size_t)jp * nx + i)), pc);
                const V dym = A::sub(pc, A::load(__ldg(ph + (size_t)k * plane + (size_t)jm * nx + i)));
                const V dzp = (k + 1 < nz) ? A::sub(A::load(__ldg(ph + c + plane)), pc) : A::zero();
                const V dzm = (k > 0) ? A::sub(pc, A::load(__ldg(ph + c - plane))) : A::zero();
                V lap = A::add(A::mul(cu, A::sub(dxp, dxm)), A::mul(cv, A::sub(dyp, dym)));
                lap = A::add(lap, A::sub(A::mul(cwp, dzp), A::mul(cwm, dzm)));
                const float2 bb = w.bdf[G.cell_off + c];
                V bvv;
                if (sizeof(T) == 4) bvv = *reinterpret_cast<const V *>(&bb);
                else bvv = A::zero();
                bv = A::sub(A::sub(bvv, cp), lap);
            }
            acc = A::add(acc, bv);
            val = to_T<T, A>(bv) * scale;
        }
        T *slot = reinterpret_cast<T *>(buf + (size_t)(jl >> 1) * sstride + fft_pos_nat(i, N2)) + (jl & 1);
        *slot = val;
    }
    // plane sum of this block's rows (for the singular mode), fixed reduction order
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
    fft_batch<T, -1>(buf, rows >> 1, sstride, N1, N2, twx);

    // split the two real rows and store x-modes m = 0..nx/2 in column blocks
    const int mb = G.mb, ncb = G.ncb, nxh = G.nxh;
    cx<T> *spec = reinterpret_cast<cx<T> *>(w.spec) + G.spec_off + (size_t)k * ncb * ny * mb;
    const int nout = ncb * rows * mb;
    for (int t = threadIdx.x; t < nout; t += blockDim.x) {
        const int mm = t % mb;
        const int rest = t / mb;
        const int jl = rest % rows, cb = rest / rows;
        const int m = cb * mb + mm, j = j0 + jl;
        if (m >= nxh || j >= ny) continue;
        const cx<T> *seq = buf + (size_t)(jl >> 1) * sstride;
        const cx<T> Zm = seq[fft_pos_tr(m, N1, N2)];
        const cx<T> Zc = seq[fft_pos_tr(m == 0 ? 0 : nx - m, N1, N2)];
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

template <typename T>
__global__ void __launch_bounds__(kYZThreads, sizeof(T) == 4 ? 4 : 2) k_yzfwd(Work w) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    cx<T> *buf = reinterpret_cast<cx<T> *>(smem_raw);
    const int g = find_grid(w.yzblk_start, w.ngrids, blockIdx.x);
    const GridDev &G = w.grids[g];
    const int cb = blockIdx.x - __ldg(w.yzblk_start + g);
    const int ny = G.ny, nz = G.nz, mb = G.mb, ncb = G.ncb, nxh = G.nxh;
    const int N1 = G.ny1, N2 = G.ny2, sstride = fft_seq_len(N1, N2) + 1;
    const int nslot = ny * mb;
    const cx<T> *twy = reinterpret_cast<const cx<T> *>(w.twy) + G.twy_off;
    const T *az = zarr<T>(w.z.az, w.z.azf) + G.z_off;
    const int tid = threadIdx.x, nthr = blockDim.x;

    // Thomas state d'_{k-1} of every mode of the block, in shared memory after the FFT buffer
    cx<T> *state = buf + (size_t)mb * sstride;
    for (int q = tid; q < nslot; q += nthr) state[q] = {(T)0, (T)0};

    for (int k = 0; k < nz; ++k) {
        cx<T> *pl = reinterpret_cast<cx<T> *>(w.spec) + G.spec_off + ((size_t)k * ncb + cb) * nslot;
        const T *tabk = reinterpret_cast<const T *>(w.tab) + G.tab_off + ((size_t)k * ncb + cb) * nslot;
        for (int t = tid; t < nslot; t += nthr) {
            const int mm = t % mb, j = t / mb;
            cx<T> v = {(T)0, (T)0};
            if (cb * mb + mm < nxh) v = pl[t];
            buf[mm * sstride + fft_pos_nat(j, N2)] = v;
        }
        __syncthreads();
        fft_batch<T, -1>(buf, mb, sstride, N1, N2, twy);
        const T a = az[k];
        for (int q = tid; q < nslot; q += nthr) {
            const int mm = q % mb, sn = q / mb;
            const cx<T> rin = buf[mm * sstride + (sn / N2) * (N2 + 1) + (sn % N2)];
            const T inv = __ldg(tabk + q);
            const cx<T> dp = state[q];
            cx<T> d = {(rin.x - a * dp.x) * inv, (rin.y - a * dp.y) * inv};
            if (cb == 0 && q == 0) d = rin;  // (0,0) mode: solved by k_00
            state[q] = d;
            if (cb * mb + mm < nxh) pl[q] = d;
        }
        __syncthreads();
    }
}

template <typename T>
__global__ void __launch_bounds__(kYZThreads, sizeof(T) == 4 ? 4 : 2) k_yzbwd(Work w) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    cx<T> *buf = reinterpret_cast<cx<T> *>(smem_raw);
    const int g = find_grid(w.yzblk_start, w.ngrids, blockIdx.x);
    const GridDev &G = w.grids[g];
    const int cb = blockIdx.x - __ldg(w.yzblk_start + g);
    const int ny = G.ny, nz = G.nz, mb = G.mb, ncb = G.ncb, nxh = G.nxh;
    const int N1 = G.ny1, N2 = G.ny2, sstride = fft_seq_len(N1, N2) + 1;
    const int nslot = ny * mb;
    const cx<T> *twy = reinterpret_cast<const cx<T> *>(w.twy) + G.twy_off;
    const T *cz = zarr<T>(w.z.cz, w.z.czf) + G.z_off;
    const int tid = threadIdx.x, nthr = blockDim.x;

    cx<T> *state = buf + (size_t)mb * sstride;  // phi_hat_{k+1} of every mode of the block
    for (int q = tid; q < nslot; q += nthr) state[q] = {(T)0, (T)0};

    for (int k = nz - 1; k >= 0; --k) {
        cx<T> *pl = reinterpret_cast<cx<T> *>(w.spec) + G.spec_off + ((size_t)k * ncb + cb) * nslot;
        const T *tabk = reinterpret_cast<const T *>(w.tab) + G.tab_off + ((size_t)k * ncb + cb) * nslot;
        const T c = cz[k];
        for (int q = tid; q < nslot; q += nthr) {
            const int mm = q % mb, sn = q / mb;
            cx<T> d = {(T)0, (T)0};
            if (cb * mb + mm < nxh) d = pl[q];
            const T cp = c * __ldg(tabk + q);
            const cx<T> nx_ = state[q];
            cx<T> ph = {d.x - cp * nx_.x, d.y - cp * nx_.y};
            if (cb == 0 && q == 0) ph = d;
            state[q] = ph;
            buf[mm * sstride + (sn / N2) * (N2 + 1) + (sn % N2)] = ph;
        }
        __syncthreads();
        fft_batch<T, +1>(buf, mb, sstride, N1, N2, twy);
        for (int t = tid; t < nslot; t += nthr) {
            const int mm = t % mb, j = t / mb;
            if (cb * mb + mm < nxh) pl[t] = buf[mm * sstride + fft_pos_nat(j, N2)];
        }
        __syncthreads();
    }
}

// ================================================================ k_00 (fp64, one CTA per grid)
template <typename T>
__global__ void __launch_bounds__(256) k_00(Work w, int first_solve) {
    extern __shared__ double rhs[];  // nz entries
    __shared__ double red[8];
    const int g = blockIdx.x;
    const GridDev &G = w.grids[g];
    const int nz = G.nz, nrb = G.nrb, zo = G.z_off;
    const double *part = w.partial + G.part_off;
    double loc = 0.0, locp = 0.0;
    bool bad = false;
    for (int k = threadIdx.x; k < nz; k += blockDim.x) {
        double S = 0.0;
        for (int r = 0; r < nrb; ++r) S += part[k * nrb + r];
        const double m = S * G.inv_nxy;  // plane mean of the right-hand side
        if (!isfinite(m)) bad = true;
        rhs[k] = m;
        loc += w.z.hz[zo + k] * m;
        if (!first_solve) {
            double P = 0.0;
            for (int r = 0; r < nrb; ++r) P += w.partial_phi[G.part_off + k * nrb + r];
            locp += w.z.hz[zo + k] * P * G.inv_nxy;
        }
    }
    if (bad) atomicOr(w.err, 1u << 6);  // IBF_ERR_NONFINITE
    __syncthreads();
    const double tot = Red<F64Arith>::sum(loc, red);
    // weighted mean of the phi being refined: the correction also removes it, so that
    // phi + delta keeps a zero weighted mean (L cannot see a constant)
    const double totp = first_solve ? 0.0 : Red<F64Arith>::sum(locp, red);
    if (threadIdx.x == 0) {
        const double mean = tot / G.sum_hz;
        if (first_solve) {
            w.mean_b[g] = mean;
            double scale = 0.0;
            for (int k = 0; k < nz; ++k) scale = fmax(scale, fabs(rhs[k]));
            // compatibility defect large compared with the plane means -> warning
            if (fabs(mean) > 1e-8 * scale && fabs(mean) > 0.0) atomicOr(w.err, 1u << 7);
        }
        // pinned Thomas: level 0 fixed to zero (inv00_0 = 0), rows 1..nz-1
        const double *az = w.z.az + zo, *cz = w.z.cz + zo, *iv = w.z.inv00 + zo;
        double d = 0.0;
        for (int k = 0; k < nz; ++k) {
            d = (rhs[k] - mean - az[k] * d) * iv[k];
            rhs[k] = d;
        }
        double nx_ = 0.0, sv = 0.0;
        for (int k = nz - 1; k >= 0; --k) {
            nx_ = rhs[k] - cz[k] * iv[k] * nx_;
            rhs[k] = nx_;
            sv += w.z.hz[zo + k] * nx_;
        }
        const double mphi = (sv + totp) / G.sum_hz;
        cx<T> *spec = reinterpret_cast<cx<T> *>(w.spec) + G.spec_off;
        const size_t stride = (size_t)G.ncb * G.ny * G.mb;
        for (int k = 0; k < nz; ++k) spec[(size_t)k * stride] = {(T)(rhs[k] - mphi), (T)0};
    }
}

// ================================================================ k_xinv
template <typename T, class A, int IMODE>
__global__ void __launch_bounds__(kXThreads, sizeof(T) == 4 ? 2 : 1) k_xinv(Work w, UserPtrs p, int use_ws) {
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
    const int mb = G.mb, ncb = G.ncb, nxh = G.nxh;
    const cx<T> *spec = reinterpret_cast<const cx<T> *>(w.spec) + G.spec_off + (size_t)k * ncb * ny * mb;
    const int npair = rows >> 1;
    const int nload = ncb * npair * mb;
    for (int t = threadIdx.x; t < nload; t += blockDim.x) {
        const int mm = t % mb;
        const int rest = t / mb;
        const int s = rest % npair, cb = rest / npair;
        const int m = cb * mb + mm;
        if (m >= nxh) continue;
        const int ja = j0 + 2 * s, jb = ja + 1;
        cx<T> A_ = {(T)0, (T)0}, B_ = {(T)0, (T)0};
        if (ja < ny) A_ = spec[((size_t)cb * ny + ja) * mb + mm];
        if (jb < ny) B_ = spec[((size_t)cb * ny + jb) * mb + mm];
        cx<T> *seq = buf + (size_t)s * sstride;
        seq[fft_pos_tr(m, N1, N2)] = {A_.x - B_.y, A_.y + B_.x};
        if (m > 0 && 2 * m < nx) seq[fft_pos_tr(nx - m, N1, N2)] = {A_.x + B_.y, B_.x - A_.y};
    }
    __syncthreads();
    const cx<T> *twx = reinterpret_cast<const cx<T> *>(w.twx) + G.twx_off;
    fft_batch<T, +1>(buf, npair, sstride, N1, N2, twx);

    const int gi = g - p.g0;
    double *phi = use_ws ? (w.phi_ws + G.cell_off) : p.out_p[gi];
    const size_t plane = (size_t)nx * ny;
    const int ncell = rows * nx;
    for (int t = threadIdx.x; t < ncell; t += blockDim.x) {
        const int jl = t / nx, i = t - jl * nx;
        const int j = j0 + jl;
        if (j >= ny) continue;
        const cx<T> z = buf[(size_t)(jl >> 1) * sstride + fft_pos_nat(i, N2)];
        const T val = (jl & 1) ? z.y : z.x;
        const size_t c = (size_t)k * plane + (size_t)j * nx + i;
        if (IMODE == IM_STORE) {
            if (sizeof(T) == 8) phi[c] = (double)val;
            else phi[c] = f32_to_f64((float)val);
        } else {
            phi[c] = A::store(A::add(A::load(phi[c]), A::from_f((float)val)));
        }
    }
}

// ================================================================ k_correct
// forward (ADJ = 0): u = u* + s rdx (phi_{i-1} - phi_i), v likewise,
//                    w_k = w*_k + s rgzf_k (phi_{k-1} - phi_k), wall faces copied.
// adjoint (ADJ = 1): g* = g_u + hz_k rdx (psi_{i-1} - psi_i), ...,
//                    w_k = g_w,k + psi_{k-1} [k>=1] - psi_k [k<=nz-1].
template <class A, int ADJ>
__global__ void __launch_bounds__(kXThreads) k_correct(Work w, UserPtrs p, int use_ws, double s) {
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
    const double *phi = use_ws ? (w.phi_ws + G.cell_off) : p.out_p[gi];
    const double *ui = p.in_u[gi], *vi = p.in_v[gi], *wi = p.in_w[gi];
    double *uo = p.out_u[gi], *vo = p.out_v[gi], *wo = p.out_w[gi];
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
    const size_t plane = (size_t)nx * ny;
    const int ncell = rows * nx;
    for (int t = threadIdx.x; t < ncell; t += blockDim.x) {
        const int jl = t / nx, i = t - jl * nx;
        const int j = j0 + jl;
        if (j >= ny) continue;
        const int im = (i == 0) ? nx - 1 : i - 1;
        const int jm = (j == 0) ? ny - 1 : j - 1;
        const size_t c = (size_t)k * plane + (size_t)j * nx + i;
        const V pc = A::load(__ldg(phi + c));
        const V pim = A::load(__ldg(phi + (size_t)k * plane + (size_t)j * nx + im));
        const V pjm = A::load(__ldg(phi + (size_t)k * plane + (size_t)jm * nx + i));
        uo[c] = A::store(A::add(A::load(ui[c]), A::mul(cu, A::sub(pim, pc))));
        vo[c] = A::store(A::add(A::load(vi[c]), A::mul(cv, A::sub(pjm, pc))));
        if (ADJ) {
            V dz = A::sub((k > 0) ? A::load(__ldg(phi + c - plane)) : A::zero(), pc);
            wo[c] = A::store(A::add(A::load(wi[c]), dz));
            if (k == nz - 1) wo[c + plane] = A::store(A::add(A::load(wi[c + plane]), pc));
        } else {
            if (k == 0) wo[c] = wi[c];
            else {
                const V pkm = A::load(__ldg(phi + c - plane));
                wo[c] = A::store(A::add(A::load(wi[c]), A::mul(cw, A::sub(pkm, pc))));
            }
            if (k == nz - 1) wo[c + plane] = wi[c + plane];
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
    const double *u = p.out_u[gi], *vv = p.out_v[gi], *ww = p.out_w[gi];
    const V cu = Coef<A>::c(G.rdx), cv = Coef<A>::c(G.rdy), cw = Coef<A>::c(w.z.rhz[G.z_off + k]);
    const size_t plane = (size_t)nx * ny;
    float mx = 0.f;
    const int ncell = rows * nx;
    for (int t = threadIdx.x; t < ncell; t += blockDim.x) {
        const int jl = t / nx, i = t - jl * nx;
        const int j = j0 + jl;
        if (j >= ny) continue;
        const int ip = (i + 1 == nx) ? 0 : i + 1;
        const int jp = (j + 1 == ny) ? 0 : j + 1;
        const size_t c = (size_t)k * plane + (size_t)j * nx + i;
        const size_t rowk = (size_t)k * plane + (size_t)j * nx;
        V d = A::mul(cu, A::sub(A::load(u[rowk + ip]), A::load(u[rowk + i])));
        d = A::add(d, A::mul(cv, A::sub(A::load(vv[(size_t)k * plane + (size_t)jp * nx + i]), A::load(vv[c]))));
        d = A::add(d, A::mul(cw, A::sub(A::load(ww[c + plane]), A::load(ww[c]))));
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

cudaError_t launch_xfwd(int mixed, int mode, const Work &w, const UserPtrs &p, int use_ws, int nblk, double s,
                        double rs, size_t smem, cudaStream_t st) {
    if (nblk <= 0) return cudaSuccess;
    if (mixed) {
        if (mode == XM_DIV) k_xfwd<float, DFArith, XM_DIV><<<grid1(nblk), kXThreads, smem, st>>>(w, p, use_ws, s, rs);
        else if (mode == XM_RESID) k_xfwd<float, DFArith, XM_RESID><<<grid1(nblk), kXThreads, smem, st>>>(w, p, use_ws, s, rs);
        else k_xfwd<float, DFArith, XM_ADJ><<<grid1(nblk), kXThreads, smem, st>>>(w, p, use_ws, s, rs);
    } else {
        if (mode == XM_DIV) k_xfwd<double, F64Arith, XM_DIV><<<grid1(nblk), kXThreads, smem, st>>>(w, p, use_ws, s, rs);
        else if (mode == XM_ADJ) k_xfwd<double, F64Arith, XM_ADJ><<<grid1(nblk), kXThreads, smem, st>>>(w, p, use_ws, s, rs);
        else return cudaErrorInvalidValue;
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
    const size_t smem = (size_t)maxnz * sizeof(double);
    if (mixed) k_00<float><<<w.ngrids, 256, smem, st>>>(w, first_solve);
    else k_00<double><<<w.ngrids, 256, smem, st>>>(w, first_solve);
    return cudaGetLastError();
}

cudaError_t launch_xinv(int mixed, int mode, const Work &w, const UserPtrs &p, int use_ws, int nblk, size_t smem,
                        cudaStream_t st) {
    if (nblk <= 0) return cudaSuccess;
    if (mixed) {
        if (mode == IM_STORE) k_xinv<float, DFArith, IM_STORE><<<grid1(nblk), kXThreads, smem, st>>>(w, p, use_ws);
        else k_xinv<float, DFArith, IM_ACCUM><<<grid1(nblk), kXThreads, smem, st>>>(w, p, use_ws);
    } else {
        k_xinv<double, F64Arith, IM_STORE><<<grid1(nblk), kXThreads, smem, st>>>(w, p, use_ws);
    }
    return cudaGetLastError();
}

cudaError_t launch_correct(int mixed, int adjoint, const Work &w, const UserPtrs &p, int use_ws, int nblk, double s,
                           cudaStream_t st) {
    if (nblk <= 0) return cudaSuccess;
    if (mixed) {
        if (adjoint) k_correct<DFArith, 1><<<grid1(nblk), kXThreads, 0, st>>>(w, p, use_ws, s);
        else k_correct<DFArith, 0><<<grid1(nblk), kXThreads, 0, st>>>(w, p, use_ws, s);
    } else {
        if (adjoint) k_correct<F64Arith, 1><<<grid1(nblk), kXThreads, 0, st>>>(w, p, use_ws, s);
        else k_correct<F64Arith, 0><<<grid1(nblk), kXThreads, 0, st>>>(w, p, use_ws, s);
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

cudaError_t set_smem_limits(int mixed, size_t xsmem, size_t yzsmem) {
    cudaError_t e = cudaSuccess;
#define IBF_ATTR(kern, bytes) \
    if (e == cudaSuccess) e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)(bytes));
    if (mixed) {
        IBF_ATTR((k_xfwd<float, DFArith, XM_DIV>), xsmem)
        IBF_ATTR((k_xfwd<float, DFArith, XM_RESID>), xsmem)
        IBF_ATTR((k_xfwd<float, DFArith, XM_ADJ>), xsmem)
        IBF_ATTR((k_xinv<float, DFArith, IM_STORE>), xsmem)
        IBF_ATTR((k_xinv<float, DFArith, IM_ACCUM>), xsmem)
        IBF_ATTR(k_yzfwd<float>, yzsmem)
        IBF_ATTR(k_yzbwd<float>, yzsmem)
    } else {
        IBF_ATTR((k_xfwd<double, F64Arith, XM_DIV>), xsmem)
        IBF_ATTR((k_xfwd<double, F64Arith, XM_ADJ>), xsmem)
        IBF_ATTR((k_xinv<double, F64Arith, IM_STORE>), xsmem)
        IBF_ATTR(k_yzfwd<double>, yzsmem)
        IBF_ATTR(k_yzbwd<double>, yzsmem)
    }
#undef IBF_ATTR
    return e;
}

}  // namespace ibf

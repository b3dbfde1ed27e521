// ibf_viscous.cu -- sm_103a kernels of the factored implicit viscous solve
// (Section "Fluid Mechanics", Eq. nstime_discr with the viscous terms advanced by
// Crank-Nicolson; Section "Fluid domain", provisional-step paragraph: the implicit
// operator split into one tridiagonal solve per direction, Thomas' algorithm, with a
// Sherman-Morrison perturbation on the periodic lines):
//
//   out = (I - beta Lz)^-1 (I - beta Ly)^-1 (I - beta Lx)^-1 rhs,  beta = alpha dt / (2 Re)
//
// for each velocity component.  On the periodic, uniform x and y lines (I - beta L)
// is circulant: its inverse -- the result the cyclic Thomas solve with the
// Sherman-Morrison correction returns -- divides Fourier coefficient m by
// 1 + beta (4/h^2) sin^2(pi m / n).  The x and y factors are therefore applied in
// the spectrum the projection's transforms already produce, and only z keeps a
// tridiagonal solve.  One component is four launches:
//   k_xfwd<XM_COPY>  x-FFT of the field (ibf_kernels.cu), spectrum in column blocks
//   k_yhelm          y-FFT, division by both factors, inverse y-FFT, in place
//   k_xinv STORE     inverse x-FFT into the plan's per-cell workspace (ibf_kernels.cu)
//   k_zhelm          Thomas along z for every (i, j) column, fp64 output.
// The z operator is the second difference of the component's own grid: cell centres
// with no-slip walls (mirror ghosts) for u and v, interior faces for w (its wall faces
// stay zero).
#include "ibf_common.cuh"
#include "ibf_viscous.h"

namespace ibf {

// Per grid (one block each): thread 0 builds the Thomas pivots of (I - beta Lz) for the
// cell-centre operator (u, v), thread 1 those of the interior-face operator (w), the
// other threads the x and y factors of k_yhelm.  Per grid and operator, at
// tab + 6 z_off + 3 op (nz+1): the sub-diagonal a_r, the pivot inverse inv_r and the
// normalised super-diagonal cp_r (nz+1 entries each), so that the forward sweep is
// y_r = (f_r - a_r y_{r-1}) inv_r and the back substitution x_r = y_r - cp_r x_{r+1}.
// fp64, with fp32 copies at the same offsets in tabf (and fxyf).
__global__ void k_helm_table(Work w, double beta, double *tab, float *tabf, const long long *fxy_off, double *fxy,
                             float *fxyf) {
    const int g = blockIdx.x, op = threadIdx.x;
    const GridDev &G = w.grids[g];
    if (op >= 2) {
        // the x and y factors 1 / (1 + beta (4/h^2) sin^2(pi m / n)) of the x-modes m < nxh
        // and the y-modes n < ny, at fxy + fxy_off[g] (nxh + ny entries)
        double *f = fxy + fxy_off[g];
        float *ff = fxyf + fxy_off[g];
        for (int t = op - 2; t < G.nxh + G.ny; t += blockDim.x - 2) {
            const bool isx = t < G.nxh;
            const int m = isx ? t : t - G.nxh;
            const double s = sinpi((double)m / (double)(isx ? G.nx : G.ny));
            const double r = isx ? G.rdx : G.rdy;
            const double v = 1.0 / (1.0 + beta * 4.0 * r * r * s * s);
            f[t] = v;
            ff[t] = (float)v;
        }
        return;
    }
    const int nz = G.nz, zo = G.z_off;
    const double *rhz = w.z.rhz + zo, *rgzf = w.z.rgzf + zo;  // 1/hz_k; 1/(zc_k - zc_{k-1}) on interior faces
    const size_t base = 6 * (size_t)zo + 3 * (size_t)op * (size_t)(nz + 1), len = (size_t)(nz + 1);
    double *a = tab + base, *inv = a + len, *cp = inv + len;
    float *af = tabf + base, *invf = af + len, *cpf = invf + len;
    const int n = op == 0 ? nz : nz - 1;
    double cprev = 0.0;
    for (int r = 0; r < n; ++r) {
        double lo, up, extra = 0.0;
        if (op == 0) {
            // centre r: neighbours across faces r and r+1; at a wall the mirror ghost
            // (minus the value) sits hz away, adding its coupling to the diagonal
            lo = r > 0 ? rhz[r] * rgzf[r] : rhz[0] * rhz[0];
            up = r < nz - 1 ? rhz[r] * rgzf[r + 1] : rhz[nz - 1] * rhz[nz - 1];
            if (r == 0) extra += lo;
            if (r == nz - 1) extra += up;
        } else {
            // interior face k = r + 1, between the centres k-1 and k
            const int k = r + 1;
            lo = rhz[k - 1] * rgzf[k];
            up = rhz[k] * rgzf[k];
        }
        const double sub = r > 0 ? -beta * lo : 0.0;
        const double sup = r < n - 1 ? -beta * up : 0.0;
        const double diag = 1.0 + beta * (lo + up + extra);
        const double iv = 1.0 / (diag - sub * cprev);
        cprev = sup * iv;
        a[r] = sub;
        inv[r] = iv;
        cp[r] = cprev;
        af[r] = (float)sub;
        invf[r] = (float)iv;
        cpf[r] = (float)cprev;
    }
}

// y-FFT, multiplication by fx_m fy_n with fx_m = 1/(1 + beta (4/dx^2) sin^2(pi m/nx))
// and fy_n likewise (tables of k_helm_table), inverse y-FFT: gb consecutive column blocks
// (cb0 .. cb0 + gb - 1, each mb x-modes) of one plane of grid g's x-spectrum, in place
// (row order in and out), as one batch of gb mb sequences so that the FFT passes have
// work for every warp when the blocks are narrow.  The x-FFT scaled by 1/(nx ny), so the
// unnormalised inverse transforms return the field.
template <typename T>
__global__ void __launch_bounds__(kYZThreads, sizeof(T) == 4 ? 4 : 1) k_yhelm(Work w, int g, int gb, const T *fxy) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const GridDev &G = w.grids[g];
    const int ncb = G.ncb, ngrp = (ncb + gb - 1) / gb;
    const int k = blockIdx.x / ngrp, cb0 = (blockIdx.x - k * ngrp) * gb;
    const int ny = G.ny, mb = G.mb, nxh = G.nxh;
    const int N1 = G.ny1, N2 = G.ny2, sstride = fft_seq_len(N1, N2) + 1;
    const FDiv fN1 = G.fny1, fN2 = G.fny2, fmb = G.fmb;
    const int nslot = ny * mb;
    const int nb = min(gb, ncb - cb0);                 // column blocks of this group
    const int nmode = min(nb * mb, nxh - cb0 * mb);    // valid x-modes of the group
    const cx<T> *twy = reinterpret_cast<const cx<T> *>(w.twy) + G.twy_off;
    cx<T> *buf = reinterpret_cast<cx<T> *>(smem_raw);
    cx<T> *pl = reinterpret_cast<cx<T> *>(w.spec) + G.spec_off + ((size_t)k * ncb + cb0) * nslot;
    const int tid = threadIdx.x, nthr = blockDim.x, ntot = gb * nslot;
    // element t of the group: column block q = t / nslot, slot t - q nslot = r mb + mm;
    // sequence s = q mb + mm (x-mode cb0 mb + s)
    for (int t = tid; t < ntot; t += nthr) {
        const int q = t / nslot, ts = t - q * nslot;
        const int r = (int)fdiv((unsigned)ts, fmb), sq = q * mb + (ts - r * mb);
        buf[sq * sstride + pos_nat(r, fN2)] = (sq < nmode) ? pl[t] : cx<T>{(T)0, (T)0};
    }
    __syncthreads();
    fft_batch<T, -1>(buf, gb * mb, sstride, N1, N2, fN1, fN2, twy);
    const T *fx = fxy + cb0 * mb, *fy = fxy + nxh;
    for (int t = tid; t < ntot; t += nthr) {
        const int q = t / nslot, ts = t - q * nslot;
        const int n = (int)fdiv((unsigned)ts, fmb), sq = q * mb + (ts - n * mb);  // y-mode n of sequence sq
        if (sq >= nmode) continue;
        const T f = fx[sq] * fy[n];
        cx<T> &v = buf[sq * sstride + pos_tr(n, N1, N2, fN1)];
        v = {v.x * f, v.y * f};
    }
    __syncthreads();
    fft_batch<T, +1>(buf, gb * mb, sstride, N1, N2, fN1, fN2, twy);
    for (int t = tid; t < ntot; t += nthr) {
        const int q = t / nslot, ts = t - q * nslot;
        const int r = (int)fdiv((unsigned)ts, fmb), sq = q * mb + (ts - r * mb);
        if (sq < nmode) pl[t] = buf[sq * sstride + pos_nat(r, fN2)];
    }
}

// Thomas along z of every (i, j) column of grid g.  Input: the x/y-solved field in the
// plan's per-cell workspace (fp32 phi_hi on the mixed path, fp64 phi_ws on the fp64
// path), planes r < n; the forward sweep overwrites it with y_r, the back substitution
// writes out (fp64).  zshift = 1: w, whose n = nz - 1 unknowns are the interior faces
// (out planes 1..nz-1; the wall faces 0 and nz are set to zero); zshift = 0: u or v.
template <typename T> struct HelmTab;
template <> struct HelmTab<float> {
    __device__ __forceinline__ static const float *get(const double *, const float *f) { return f; }
    __device__ __forceinline__ static float *ws(const Work &w) { return w.phi_hi; }
};
template <> struct HelmTab<double> {
    __device__ __forceinline__ static const double *get(const double *d, const float *) { return d; }
    __device__ __forceinline__ static double *ws(const Work &w) { return w.phi_ws; }
};

template <typename T>
__global__ void __launch_bounds__(kZHelmThreads) k_zhelm(Work w, int g, int zshift, const double *tab,
                                                         const float *tabf, double *out) {
    const GridDev &G = w.grids[g];
    const long long plane = (long long)G.nx * G.ny;
    const long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= plane) return;
    const int nz = G.nz, n = nz - zshift;
    const size_t base = 6 * (size_t)G.z_off + 3 * (size_t)zshift * (size_t)(nz + 1), len = (size_t)(nz + 1);
    const T *a = HelmTab<T>::get(tab, tabf) + base, *inv = a + len, *cp = inv + len;
    T *f = HelmTab<T>::ws(w) + G.cell_off + c;
    T y = (T)0;
#pragma unroll 4
    for (int r = 0; r < n; ++r) {
        y = (f[r * plane] - a[r] * y) * inv[r];
        f[r * plane] = y;
    }
    T x = (T)0;
#pragma unroll 4
    for (int r = n - 1; r >= 0; --r) {
        x = f[r * plane] - cp[r] * x;
        out[(r + zshift) * plane + c] = (double)x;
    }
    if (zshift) {
        out[c] = 0.0;
        out[nz * plane + c] = 0.0;
    }
}

cudaError_t launch_helm_table(const Work &w, int ngrids, double beta, double *tab, float *tabf,
                              const long long *fxy_off, double *fxy, float *fxyf, cudaStream_t st) {
    if (ngrids <= 0) return cudaSuccess;
    k_helm_table<<<ngrids, 128, 0, st>>>(w, beta, tab, tabf, fxy_off, fxy, fxyf);
    return cudaGetLastError();
}

cudaError_t launch_yhelm(int mixed, const Work &w, int g, int nblk, int gb, const double *fxy, const float *fxyf,
                         size_t smem, cudaStream_t st) {
    if (nblk <= 0) return cudaSuccess;
    if (mixed) k_yhelm<float><<<nblk, kYZThreads, smem, st>>>(w, g, gb, fxyf);
    else k_yhelm<double><<<nblk, kYZThreads, smem, st>>>(w, g, gb, fxy);
    return cudaGetLastError();
}

cudaError_t launch_zhelm(int mixed, const Work &w, int g, long long ncol, int zshift, const double *tab,
                         const float *tabf, double *out, cudaStream_t st) {
    if (ncol <= 0) return cudaSuccess;
    const unsigned nb = (unsigned)((ncol + kZHelmThreads - 1) / kZHelmThreads);
    if (mixed) k_zhelm<float><<<nb, kZHelmThreads, 0, st>>>(w, g, zshift, tab, tabf, out);
    else k_zhelm<double><<<nb, kZHelmThreads, 0, st>>>(w, g, zshift, tab, tabf, out);
    return cudaGetLastError();
}

cudaError_t set_smem_limits_visc(int mixed) {
    return mixed ? set_smem_cap((const void *)k_yhelm<float>) : set_smem_cap((const void *)k_yhelm<double>);
}

}  // namespace ibf

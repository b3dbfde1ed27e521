// ibf_yz.cu -- sm_103a kernels along y and z: the y-FFT fused with the Thomas
// sweeps of every horizontal mode (k_yzfwd / k_yzbwd), the singular (0,0) mode in
// fp64 (k_00), and the per-plan pivot table (k_build_table).  See ibf_kernels.cu
// for the data flow of one solve.
#include "ibf_common.cuh"

#include <type_traits>

namespace ibf {

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

// DCT-II post-twiddle of the FFT V (in place, FFT output order) of every Makhoul-
// reordered sequence of a column block: with P = W^n V_n, Q = conj(W^n) V_{N-n},
// W = exp(-i pi/(2N)), the coefficients are X_n = (P + Q)/2 and X_{N-n} = i (P - Q)/2
// (complex-linear, so it holds for complex columns); X_0 = V_0.  Ends synchronised.
template <typename T>
__device__ __forceinline__ void dct_post(cx<T> *buf, int nseq, int sstride, int N, int N1, int N2,
                                         const FDiv &fN1, const cx<T> *W) {
    const int half = N >> 1;
    for (int t = threadIdx.x; t < nseq * half; t += blockDim.x) {
        const int sq = t / half, n = t - sq * half + 1;
        cx<T> *seq = buf + sq * sstride;
        const int pa = pos_tr(n, N1, N2, fN1), pb = pos_tr(N - n, N1, N2, fN1);
        const cx<T> a = seq[pa], b = seq[pb], w = W[n];
        const cx<T> P = {w.x * a.x - w.y * a.y, w.x * a.y + w.y * a.x};
        const cx<T> Q = {w.x * b.x + w.y * b.y, w.x * b.y - w.y * b.x};
        if (pa == pb) {  // n = N/2
            seq[pa] = {(P.x + Q.x) * (T)0.5, (P.y + Q.y) * (T)0.5};
        } else {
            seq[pa] = {(P.x + Q.x) * (T)0.5, (P.y + Q.y) * (T)0.5};
            seq[pb] = {(Q.y - P.y) * (T)0.5, (P.x - Q.x) * (T)0.5};
        }
    }
    __syncthreads();
}

// Inverse of dct_post (DCT-III input stage, in place): V_n = conj(W^n)(X_n - i X_{N-n}),
// V_{N-n} = W^n (X_n + i X_{N-n}); V_0 = X_0.  An unscaled inverse FFT of V followed by
// the un-reordering returns the sequence whose DCT-II divided by N was X.  Ends synchronised.
template <typename T>
__device__ __forceinline__ void dct_pre(cx<T> *buf, int nseq, int sstride, int N, int N1, int N2,
                                        const FDiv &fN1, const cx<T> *W) {
    const int half = N >> 1;
    for (int t = threadIdx.x; t < nseq * half; t += blockDim.x) {
        const int sq = t / half, n = t - sq * half + 1;
        cx<T> *seq = buf + sq * sstride;
        const int pa = pos_tr(n, N1, N2, fN1), pb = pos_tr(N - n, N1, N2, fN1);
        const cx<T> a = seq[pa], b = seq[pb], w = W[n];
        const cx<T> d = {a.x + b.y, a.y - b.x};  // X_n - i X_{N-n}
        const cx<T> e = {a.x - b.y, a.y + b.x};  // X_n + i X_{N-n}
        seq[pa] = {w.x * d.x + w.y * d.y, w.x * d.y - w.y * d.x};
        if (pa != pb) seq[pb] = {w.x * e.x - w.y * e.y, w.x * e.y + w.y * e.x};
    }
    __syncthreads();
}

// y-FFT + Thomas forward elimination of one column block, sweeping k = 0..nz-1.
// Shared memory: kYZStages x [FFT buffer (mb padded sequences) | pivot chunk], then the
// Thomas state d'_{k-1} of every mode of the block.  Plane k+1 (spectrum and pivots)
// is copied with cp.async while plane k is transformed and eliminated.
template <typename T, bool W>
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
    const int wall_y = W ? G.wall_y : 0;
    const cx<T> *dcty = reinterpret_cast<const cx<T> *>(w.twy) + G.dcty_off;
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
                cx<T> *dst = fb + mm * sstride + pos_nat(wall_y ? dct_perm(j, ny) : j, fN2);
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
        if (wall_y) dct_post<T>(buf, mb, sstride, ny, N1, N2, fN1, dcty);
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
template <typename T, bool W>
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
    const int wall_y = W ? G.wall_y : 0;
    const cx<T> *dcty = reinterpret_cast<const cx<T> *>(w.twy) + G.dcty_off;
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
        if (wall_y) dct_pre<T>(buf, mb, sstride, ny, N1, N2, fN1, dcty);
        fft_batch<T, +1>(buf, mb, sstride, N1, N2, fN1, fN2, twy);
        cx<T> *pl = spec + ((size_t)k * ncb + cb) * nslot;
        for (int t = tid; t < nslot; t += nthr) {
            const int j = (int)fdiv((unsigned)t, fmb), mm = t - j * mb;
            if (mm < nvalid) pl[t] = buf[mm * sstride + pos_nat(wall_y ? dct_perm(j, ny) : j, fN2)];
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

// Pivots of every mode's tridiagonal system (fp64 arithmetic, stored as T):
// inv_k = 1/(bz_k + lambda - az_k c'_{k-1}),  c'_k = cz_k inv_k,  bz_k = -(az_k + cz_k),
// lambda = -4/dx^2 sin^2(pi m/nx) - 4/dy^2 sin^2(pi n/ny), with pi m/(2 nx), pi n/(2 ny)
// in a wall-bounded direction.
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
        // eigenvalues of the 1-D second difference: periodic (DFT) or Neumann (DCT-II) basis
        const double sx = sinpi((double)m / (G.wall_x ? 2 * G.nx : G.nx));
        const double sy = sinpi((double)n / (G.wall_y ? 2 * ny : ny));
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
cudaError_t launch_yzfwd(int mixed, const Work &w, int nblk, size_t smem, cudaStream_t st) {
    if (mixed) {
        if (w.walls) k_yzfwd<float, true><<<grid1(nblk), kYZThreads, smem, st>>>(w);
        else k_yzfwd<float, false><<<grid1(nblk), kYZThreads, smem, st>>>(w);
    } else {
        if (w.walls) k_yzfwd<double, true><<<grid1(nblk), kYZThreads, smem, st>>>(w);
        else k_yzfwd<double, false><<<grid1(nblk), kYZThreads, smem, st>>>(w);
    }
    return cudaGetLastError();
}

cudaError_t launch_yzbwd(int mixed, const Work &w, int nblk, size_t smem, cudaStream_t st) {
    if (mixed) {
        if (w.walls) k_yzbwd<float, true><<<grid1(nblk), kYZThreads, smem, st>>>(w);
        else k_yzbwd<float, false><<<grid1(nblk), kYZThreads, smem, st>>>(w);
    } else {
        if (w.walls) k_yzbwd<double, true><<<grid1(nblk), kYZThreads, smem, st>>>(w);
        else k_yzbwd<double, false><<<grid1(nblk), kYZThreads, smem, st>>>(w);
    }
    return cudaGetLastError();
}

cudaError_t launch_k00(const Work &w, int mixed, int first_solve, int maxnz, cudaStream_t st) {
    const size_t smem = (size_t)10 * (maxnz + 1) * sizeof(double);
    if (mixed) k_00<float><<<w.ngrids, 256, smem, st>>>(w, first_solve);
    else k_00<double><<<w.ngrids, 256, smem, st>>>(w, first_solve);
    return cudaGetLastError();
}

cudaError_t launch_build_table(int mixed, const Work &w, int nblk, cudaStream_t st) {
    if (mixed) k_build_table<float><<<grid1(nblk), 256, 0, st>>>(w);
    else k_build_table<double><<<grid1(nblk), 256, 0, st>>>(w);
    return cudaGetLastError();
}

cudaError_t set_smem_limits_yz(int mixed) {
    cudaError_t e = cudaSuccess;
    auto set = [&](const void *fn) {
        if (e == cudaSuccess) e = set_smem_cap(fn);
    };
    auto set_all = [&](auto wtag) {
        constexpr bool W = decltype(wtag)::value;
        if (mixed) {
            set((const void *)k_yzfwd<float, W>);
            set((const void *)k_yzbwd<float, W>);
        } else {
            set((const void *)k_yzfwd<double, W>);
            set((const void *)k_yzbwd<double, W>);
        }
    };
    set_all(std::false_type{});
    set_all(std::true_type{});
    if (mixed) set((const void *)k_00<float>);
    else set((const void *)k_00<double>);
    return e;
}

}  // namespace ibf

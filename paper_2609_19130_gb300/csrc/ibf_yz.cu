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

// ---------------------------------------------------------------- pipelined forms
// Mixed path, one x-mode per column block (mb = 1), periodic y.  A single sequence's
// two-level FFT is 32 tasks per pass, so in the plain streaming kernels one warp
// transforms each plane while the other three wait at the barriers.  Here warp 0 only
// transforms and warps 1-3 run the Thomas sweep and the copies of neighbouring planes
// in the same interval, one __syncthreads per plane:
//   forward,  iteration it: warp 0 FFT of plane it;  warps 1-3 sweep plane it-1, copy plane it+1
//   backward, iteration it: warp 0 inverse FFT of plane it-1;  warps 1-3 back-substitute
//             plane it (in place in its FFT buffer), store plane it-2, copy plane it+1
// (backward planes counted from the top).  Every slot is handled by the same warp-1-3
// thread in the copies, the sweep and the store, so that thread alone reads what it
// copied; what warp 0 transformed is read after the barrier that ends its iteration.
// Shared memory (yz_pipe_smem): forward kPipeF x [FFT buffer | pivot chunk] + state;
// backward kPipeB FFT buffers + 2 pivot chunks + state.
constexpr int kPipeT = kYZThreads - 32;  // sweep / copy threads

__device__ __forceinline__ void fft1_warp_fwd(cx<float> *buf, int sstride, int N1, int N2, const FDiv &fN1,
                                              const FDiv &fN2, const cx<float> *tw, int lane) {
    fft_col_pass<float, -1>(buf, 1, sstride, N1, N2, fN2, tw, lane, 32);
    __syncwarp();
    fft_row_pass<float, -1>(buf, 1, sstride, N1, N2, fN1, tw, lane, 32);
    __syncwarp();
}
// the same transform of a plane copied dense (row stride N2) into a buffer of the padded size
__device__ __noinline__ void fft1_warp_fwd_dense(cx<float> *buf, int sstride, int N1, int N2, const FDiv fN1,
                                                 const cx<float> *tw, int lane) {
    fft_col_pass_dense_in<float, -1>(buf, N1, N2, tw, lane);
    __syncwarp();
    fft_row_pass<float, -1>(buf, 1, sstride, N1, N2, fN1, tw, lane, 32);
    __syncwarp();
}
__device__ __forceinline__ void fft1_warp_inv(cx<float> *buf, int sstride, int N1, int N2, const FDiv &fN1,
                                              const FDiv &fN2, const cx<float> *tw, int lane) {
    fft_row_pass<float, +1>(buf, 1, sstride, N1, N2, fN1, tw, lane, 32);
    __syncwarp();
    fft_col_pass<float, +1>(buf, 1, sstride, N1, N2, fN2, tw, lane, 32);
    __syncwarp();
}

__device__ void yzfwd_pipe(const Work &w, const GridDev &G, int cb, unsigned char *smem) {
    const int ny = G.ny, nz = G.nz, ncb = G.ncb;
    const int N1 = G.ny1, N2 = G.ny2, sstride = fft_seq_len(N1, N2) + 1;
    const FDiv fN1 = G.fny1, fN2 = G.fny2;
    const size_t stage = pipe_align16((size_t)sstride * 8 + (size_t)ny * 4);
    auto fb = [&](int i) { return reinterpret_cast<cx<float> *>(smem + (size_t)(i % kPipeF) * stage); };
    auto tb = [&](int i) { return reinterpret_cast<float *>(smem + (size_t)(i % kPipeF) * stage + (size_t)sstride * 8); };
    cx<float> *state = reinterpret_cast<cx<float> *>(smem + (size_t)kPipeF * stage);
    const cx<float> *spec = reinterpret_cast<const cx<float> *>(w.spec) + G.spec_off;
    cx<float> *specw = reinterpret_cast<cx<float> *>(w.spec) + G.spec_off;
    const float *tab = reinterpret_cast<const float *>(w.tab) + G.tab_off;
    const cx<float> *twy = reinterpret_cast<const cx<float> *>(w.twy) + G.twy_off;
    const float *az = w.z.azf + G.z_off;
    const int tid = threadIdx.x, tt = tid - 32;
    const bool fw = tid < 32;
    auto issue = [&](int k) {  // spectrum and pivots of plane k into ring entry k
        if (k < nz) {
            cx<float> *f = fb(k);
            float *t = tb(k);
            const cx<float> *src = spec + ((size_t)k * ncb + cb) * ny;
            const float *tsrc = tab + ((size_t)k * ncb + cb) * ny;
            for (int j = tt; j < ny; j += kPipeT) {
                cp_async<8>(f + pos_nat(j, fN2), src + j);
                cp_async<4>(t + j, tsrc + j);
            }
        }
        cp_async_commit();
    };
    if (!fw) {
        for (int q = tt; q < ny; q += kPipeT) state[q] = {0.f, 0.f};
        issue(0);
        cp_async_wait<0>();
    }
    __syncthreads();
    for (int it = 0; it <= nz; ++it) {
        if (fw) {
            if (it < nz) fft1_warp_fwd(fb(it), sstride, N1, N2, fN1, fN2, twy, tid);
        } else {
            issue(it + 1);
            if (it >= 1) {
                const int k = it - 1;
                const cx<float> *buf = fb(k);
                const float *t = tb(k);
                cx<float> *pl = specw + ((size_t)k * ncb + cb) * ny;
                const float a = az[k];
                for (int q = tt; q < ny; q += kPipeT) {
                    const cx<float> rin = buf[pos_nat(q, fN2)];
                    const float inv = t[q];
                    const cx<float> dp = state[q];
                    cx<float> d = {(rin.x - a * dp.x) * inv, (rin.y - a * dp.y) * inv};
                    if (cb == 0 && q == 0) d = rin;  // (0,0) mode: solved by k_00
                    state[q] = d;
                    pl[q] = d;
                }
            }
            cp_async_wait<0>();  // plane it+1 is in its ring entry (this thread's copies)
        }
        __syncthreads();
    }
}

__device__ void yzbwd_pipe(const Work &w, const GridDev &G, int cb, unsigned char *smem) {
    const int ny = G.ny, nz = G.nz, ncb = G.ncb;
    const int N1 = G.ny1, N2 = G.ny2, sstride = fft_seq_len(N1, N2) + 1;
    const FDiv fN1 = G.fny1, fN2 = G.fny2;
    const size_t fstage = pipe_align16((size_t)sstride * 8), tstage = pipe_align16((size_t)ny * 4);
    auto fb = [&](int i) { return reinterpret_cast<cx<float> *>(smem + (size_t)(i % kPipeB) * fstage); };
    auto tb = [&](int i) { return reinterpret_cast<float *>(smem + kPipeB * fstage + (size_t)(i % 2) * tstage); };
    cx<float> *state = reinterpret_cast<cx<float> *>(smem + kPipeB * fstage + 2 * tstage);
    cx<float> *spec = reinterpret_cast<cx<float> *>(w.spec) + G.spec_off;
    const float *tab = reinterpret_cast<const float *>(w.tab) + G.tab_off;
    const cx<float> *twy = reinterpret_cast<const cx<float> *>(w.twy) + G.twy_off;
    const float *cz = w.z.czf + G.z_off;
    const int tid = threadIdx.x, tt = tid - 32;
    const bool fw = tid < 32;
    auto plane_of = [&](int i) { return nz - 1 - i; };  // i-th plane from the top
    auto issue = [&](int i) {  // d' (slot q to the FFT position of slot q) and pivots of plane i
        if (i < nz) {
            const int k = plane_of(i);
            cx<float> *f = fb(i);
            float *t = tb(i);
            const cx<float> *src = spec + ((size_t)k * ncb + cb) * ny;
            const float *tsrc = tab + ((size_t)k * ncb + cb) * ny;
            for (int q = tt; q < ny; q += kPipeT) {
                cp_async<8>(f + pos_nat(q, fN2), src + q);
                cp_async<4>(t + q, tsrc + q);
            }
        }
        cp_async_commit();
    };
    // the (0,0) mode's solution (k_00) for slot 0 of block 0, loaded one plane ahead
    const bool own00 = cb == 0 && tt == 0;
    double s00n = own00 ? w.sol00[G.z_off + plane_of(0)] : 0.0;
    if (!fw) {
        for (int q = tt; q < ny; q += kPipeT) state[q] = {0.f, 0.f};
        issue(0);
        cp_async_wait<0>();
    }
    __syncthreads();
    for (int it = 0; it <= nz + 1; ++it) {
        if (fw) {
            if (it >= 1 && it <= nz) fft1_warp_inv(fb(it - 1), sstride, N1, N2, fN1, fN2, twy, tid);
        } else {
            issue(it + 1);
            if (it < nz) {  // back substitution of plane it, in place in its FFT buffer
                const int k = plane_of(it);
                cx<float> *buf = fb(it);
                const float *t = tb(it);
                const float c = cz[k];
                const double s00 = s00n;
                if (own00 && it + 1 < nz) s00n = w.sol00[G.z_off + plane_of(it + 1)];
                for (int q = tt; q < ny; q += kPipeT) {
                    const int pos = pos_nat(q, fN2);
                    const cx<float> d = buf[pos];
                    const float cp = c * t[q];
                    const cx<float> nx_ = state[q];
                    cx<float> ph = {d.x - cp * nx_.x, d.y - cp * nx_.y};
                    if (cb == 0 && q == 0) ph = {(float)s00, 0.f};  // (0,0): k_00's solution
                    state[q] = ph;
                    buf[pos] = ph;
                }
            }
            if (it >= 2) {  // store plane it-2, transformed by warp 0 in the last iteration
                const int k = plane_of(it - 2);
                const cx<float> *buf = fb(it - 2);
                cx<float> *pl = spec + ((size_t)k * ncb + cb) * ny;
                for (int j = tt; j < ny; j += kPipeT) pl[j] = buf[pos_nat(j, fN2)];
            }
            cp_async_wait<0>();
        }
        __syncthreads();
    }
}

// ---------------------------------------------------------------- round-based forms
// Mixed path, one x-mode per column block, periodic y, even ny (the benchmark's shape).
// The planes of the column block go in rounds of kBulkPlanes: in round r one thread
// issues bulk asynchronous copies (cp.async.bulk, completed on an mbarrier per buffer)
// of round r+1's planes into the other of two buffer sets, while
//   forward:  warps 0..kBulkPlanes-1 each transform one plane of round r (the column
//             pass reads the dense copy and writes the padded FFT layout in place), then all threads run
//             the Thomas forward step of the round's planes in order, each thread on fixed
//             slots, the state d'_{k-1} in registers within the round;
//   backward: all threads back-substitute the round's planes in order (each thread reads
//             its slots of a plane's dense copy, a barrier, then writes phi_hat in the
//             padded layout of the same buffer), then warps 0..kBulkPlanes-1 each
//             inverse-transform one plane and store it.
// kBulkPlanes FFT warps per CTA and four CTAs per SM keep twelve plane transforms in
// flight per SM (the one-warp transform of a plane is latency-bound), and the copies of
// the next round overlap the current one.  Waits on the copies give up after
// kBulkWaitLimit polls and set IBF_ERR_TIMEOUT.
constexpr int kBulkSlots = 1024 / kYZThreads;  // slots per thread (ny <= 1024)

// After a copy of round r was not seen within the wait limit: report IBF_ERR_TIMEOUT and
// let the copies of round r+1, already issued, land (bounded) before the CTA exits.
__device__ __forceinline__ void bulk_lost_cleanup(const Work &w, unsigned long long *bar, int r, int nround, int nz,
                                                  int tid) {
    if (tid != 0) return;
    atomicOr(w.err, 1u << 5);  // IBF_ERR_TIMEOUT
    if (r + 1 < nround)
        for (int f = 0; f < kBulkPlanes && (r + 1) * kBulkPlanes + f < nz; ++f)
            mbar_wait_bounded(bar + ((r + 1) & 1) * kBulkPlanes + f, (unsigned)((r + 1) >> 1) & 1u, kBulkWaitLimit);
}

// The Thomas forward step of one round's planes (yzfwd_bulk), in a function of its own so
// that its pointers and the round's loads are not live across the transforms, which need
// the whole 128-register budget.
__device__ __noinline__ bool yzfwd_bulk_sweep(const Work &w, const GridDev &G, int cb, unsigned char *smem, int r,
                                             bool lost) {
    const int ny = G.ny, nz = G.nz, ncb = G.ncb;
    const int sstride = fft_seq_len(G.ny1, G.ny2) + 1;
    const FDiv fN2 = G.fny2;
    const size_t sb = pipe_align16((size_t)max(sstride, ny) * 8);
    auto buf = [&](int set, int f) { return reinterpret_cast<cx<float> *>(smem + (size_t)(set * kBulkPlanes + f) * sb); };
    cx<float> *specw = reinterpret_cast<cx<float> *>(w.spec) + G.spec_off;
    const float *tab = reinterpret_cast<const float *>(w.tab) + G.tab_off;
    const float *az = w.z.azf + G.z_off;
    const int tid = threadIdx.x;
    // All of the round's global loads first (the state and the pivots of every
    // plane), so that the sweep waits for memory once per round.
    cx<float> st[kBulkSlots];
    float inv[kBulkPlanes][kBulkSlots];
#pragma unroll
    for (int i = 0; i < kBulkSlots; ++i) {
        const int q = tid + i * kYZThreads;
        st[i] = (r > 0 && q < ny) ? specw[((size_t)(r * kBulkPlanes - 1) * ncb + cb) * ny + q] : cx<float>{0.f, 0.f};
    }
#pragma unroll
    for (int f = 0; f < kBulkPlanes; ++f) {
        const int k = min(r * kBulkPlanes + f, nz - 1);
        const float *t = tab + ((size_t)k * ncb + cb) * ny;
#pragma unroll
        for (int i = 0; i < kBulkSlots; ++i) {
            const int q = tid + i * kYZThreads;
            inv[f][i] = q < ny ? __ldg(t + q) : 0.f;
        }
    }
    // the round's transforms are done (and every thread's loads above are in flight)
    // once all threads pass this barrier; a lost copy stops the column block
    if (__syncthreads_or(lost)) return true;
#pragma unroll
    for (int f = 0; f < kBulkPlanes; ++f) {
        const int k = r * kBulkPlanes + f;
        if (k < nz) {
            const cx<float> *b = buf(r & 1, f);
            cx<float> *pl = specw + ((size_t)k * ncb + cb) * ny;
            const float a = az[k];
#pragma unroll
            for (int i = 0; i < kBulkSlots; ++i) {
                const int q = tid + i * kYZThreads;
                if (q < ny) {
                    const cx<float> rin = b[pos_nat(q, fN2)];
                    cx<float> d = {(rin.x - a * st[i].x) * inv[f][i], (rin.y - a * st[i].y) * inv[f][i]};
                    if (cb == 0 && q == 0) d = rin;  // (0,0) mode: solved by k_00
                    st[i] = d;
                    pl[q] = d;
                }
            }
        }
    }
    return false;
}

__device__ void yzfwd_bulk(const Work &w, const GridDev &G, int cb, unsigned char *smem) {
    const int ny = G.ny, nz = G.nz, ncb = G.ncb;
    const int N1 = G.ny1, N2 = G.ny2, sstride = fft_seq_len(N1, N2) + 1;
    const FDiv fN1 = G.fny1;
    const size_t sb = pipe_align16((size_t)max(sstride, ny) * 8);
    auto buf = [&](int set, int f) { return reinterpret_cast<cx<float> *>(smem + (size_t)(set * kBulkPlanes + f) * sb); };
    unsigned long long *bar = reinterpret_cast<unsigned long long *>(smem + 2 * kBulkPlanes * sb);
    const cx<float> *spec = reinterpret_cast<const cx<float> *>(w.spec) + G.spec_off;
    const cx<float> *twy = reinterpret_cast<const cx<float> *>(w.twy) + G.twy_off;
    const float *tab = reinterpret_cast<const float *>(w.tab) + G.tab_off;
    const bool tab_pf = ((G.tab_off | ny) & 3) == 0;  // pivot rows 16-byte aligned
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int nround = (nz + kBulkPlanes - 1) / kBulkPlanes;
    const unsigned bytes = (unsigned)ny * 8u;
    if (tid == 0) {
        for (int i = 0; i < 2 * kBulkPlanes; ++i) mbar_init(bar + i, 1);
        mbar_init_fence();
    }
    __syncthreads();
    auto issue = [&](int r) {  // thread 0: the planes of round r into set r & 1
        for (int f = 0; f < kBulkPlanes; ++f) {
            const int k = r * kBulkPlanes + f;
            if (k >= nz) break;
            if (w.fault_lose_copy && r == 1 && f == 0) continue;  // test hook: this copy never arrives
            unsigned long long *b = bar + (r & 1) * kBulkPlanes + f;
            mbar_arrive_expect_tx(b, bytes);
            bulk_g2s(buf(r & 1, f), spec + ((size_t)k * ncb + cb) * ny, bytes, b);
            // the plane's pivots, read by the sweep of round r: into L2 meanwhile
            if (tab_pf) bulk_prefetch_l2(tab + ((size_t)k * ncb + cb) * ny, (unsigned)ny * 4u);
        }
    };
    if (tid == 0) issue(0);
    bool lost = false;
    for (int r = 0; r < nround; ++r) {
        if (tid == 0 && r + 1 < nround) {
            fence_proxy_async_smem();
            issue(r + 1);
        }
        if (warp < kBulkPlanes) {
            const int k = r * kBulkPlanes + warp;
            if (k < nz) {
                if (mbar_wait_bounded(bar + (r & 1) * kBulkPlanes + warp, (unsigned)(r >> 1) & 1u, kBulkWaitLimit)) {
                    fft1_warp_fwd_dense(buf(r & 1, warp), sstride, N1, N2, fN1, twy, lane);
                }
                else
                    lost = true;
            }
        }
        // the sweep reads back, as the Thomas state, what each thread stored for the last
        // plane of the previous round (rather than holding it across the transforms); its
        // loads are issued before the barrier that ends the transforms.  A lost copy stops
        // the column block: the error is reported, nothing more is waited on
        if (yzfwd_bulk_sweep(w, G, cb, smem, r, lost)) {
            bulk_lost_cleanup(w, bar, r, nround, nz, tid);
            return;
        }
        fence_proxy_async_smem();  // this thread's reads of the set before its next copies
        __syncthreads();
    }
    if (tid == 0)
        for (int i = 0; i < 2 * kBulkPlanes; ++i) mbar_inval(bar + i);
}

__device__ __noinline__ void fft1_warp_inv_call(cx<float> *buf, int sstride, int N1, int N2, const FDiv fN1,
                                                const FDiv fN2, const cx<float> *tw, int lane) {
    fft1_warp_inv(buf, sstride, N1, N2, fN1, fN2, tw, lane);
}

__device__ void yzbwd_bulk(const Work &w, const GridDev &G, int cb, unsigned char *smem) {
    const int ny = G.ny, nz = G.nz, ncb = G.ncb;
    const int N1 = G.ny1, N2 = G.ny2, sstride = fft_seq_len(N1, N2) + 1;
    const FDiv fN1 = G.fny1, fN2 = G.fny2;
    const size_t sb = pipe_align16((size_t)max(sstride, ny) * 8);
    auto buf = [&](int set, int f) { return reinterpret_cast<cx<float> *>(smem + (size_t)(set * kBulkPlanes + f) * sb); };
    unsigned long long *bar = reinterpret_cast<unsigned long long *>(smem + 2 * kBulkPlanes * sb);
    cx<float> *spec = reinterpret_cast<cx<float> *>(w.spec) + G.spec_off;
    const float *tab = reinterpret_cast<const float *>(w.tab) + G.tab_off;
    const bool tab_pf = ((G.tab_off | ny) & 3) == 0;  // pivot rows 16-byte aligned
    const cx<float> *twy = reinterpret_cast<const cx<float> *>(w.twy) + G.twy_off;
    const float *cz = w.z.czf + G.z_off;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int nround = (nz + kBulkPlanes - 1) / kBulkPlanes;
    const unsigned bytes = (unsigned)ny * 8u;
    if (tid == 0) {
        for (int i = 0; i < 2 * kBulkPlanes; ++i) mbar_init(bar + i, 1);
        mbar_init_fence();
    }
    __syncthreads();
    auto issue = [&](int r) {  // planes counted from the top: i = r kBulkPlanes + f -> k = nz - 1 - i
        for (int f = 0; f < kBulkPlanes; ++f) {
            const int i = r * kBulkPlanes + f;
            if (i >= nz) break;
            const int k = nz - 1 - i;
            unsigned long long *b = bar + (r & 1) * kBulkPlanes + f;
            mbar_arrive_expect_tx(b, bytes);
            bulk_g2s(buf(r & 1, f), spec + ((size_t)k * ncb + cb) * ny, bytes, b);
            // the plane's pivots, read at the start of round r: into L2 meanwhile
            if (tab_pf) bulk_prefetch_l2(tab + ((size_t)k * ncb + cb) * ny, (unsigned)ny * 4u);
        }
    };
    if (tid == 0) issue(0);
    cx<float> st[kBulkSlots];  // phi_hat_{k+1} of this thread's slots
#pragma unroll
    for (int i = 0; i < kBulkSlots; ++i) st[i] = {0.f, 0.f};
    for (int r = 0; r < nround; ++r) {
        if (tid == 0 && r + 1 < nround) {
            fence_proxy_async_smem();
            issue(r + 1);
        }
        // the pivots (times cz_k) of every plane of the round, loaded before any wait
        float cp[kBulkPlanes][kBulkSlots];
        float s00[kBulkPlanes];
#pragma unroll
        for (int f = 0; f < kBulkPlanes; ++f) {
            const int k = max(nz - 1 - (r * kBulkPlanes + f), 0);
            const float *t = tab + ((size_t)k * ncb + cb) * ny;
            const float c = cz[k];
#pragma unroll
            for (int i = 0; i < kBulkSlots; ++i) {
                const int q = tid + i * kYZThreads;
                cp[f][i] = q < ny ? c * __ldg(t + q) : 0.f;
            }
            s00[f] = (cb == 0 && tid == 0) ? (float)w.sol00[G.z_off + k] : 0.f;
        }
#pragma unroll
        for (int f = 0; f < kBulkPlanes; ++f) {
            const int i0 = r * kBulkPlanes + f;
            if (i0 >= nz) break;
            // each thread reads its slots of the plane's dense copy once its wait has seen
            // the copy land; one barrier then both ends the reads (the padded layout of the
            // same buffer may be written) and tells every thread whether a copy was lost
            const bool arrived =
                mbar_wait_bounded(bar + (r & 1) * kBulkPlanes + f, (unsigned)(r >> 1) & 1u, kBulkWaitLimit);
            cx<float> *b = buf(r & 1, f);
            cx<float> dv[kBulkSlots];
#pragma unroll
            for (int i = 0; i < kBulkSlots; ++i) {
                const int q = tid + i * kYZThreads;
                dv[i] = (arrived && q < ny) ? b[q] : cx<float>{0.f, 0.f};
            }
            // a lost copy stops the column block: the error is reported, nothing more is waited on
            if (__syncthreads_or(!arrived)) {
                bulk_lost_cleanup(w, bar, r, nround, nz, tid);
                return;
            }
#pragma unroll
            for (int i = 0; i < kBulkSlots; ++i) {
                const int q = tid + i * kYZThreads;
                if (q < ny) {
                    cx<float> ph = {dv[i].x - cp[f][i] * st[i].x, dv[i].y - cp[f][i] * st[i].y};
                    if (cb == 0 && q == 0) ph = {s00[f], 0.f};  // (0,0): k_00's solution
                    st[i] = ph;
                    b[pos_nat(q, fN2)] = ph;
                }
            }
        }
        __syncthreads();
        if (warp < kBulkPlanes) {
            const int i0 = r * kBulkPlanes + warp;
            if (i0 < nz) {
                const int k = nz - 1 - i0;
                cx<float> *b = buf(r & 1, warp);
                fft1_warp_inv_call(b, sstride, N1, N2, fN1, fN2, twy, lane);
                cx<float> *pl = spec + ((size_t)k * ncb + cb) * ny;
                for (int j = lane; j < ny; j += 32) pl[j] = b[pos_nat(j, fN2)];
            }
        }
        fence_proxy_async_smem();
        __syncthreads();
    }
    if (tid == 0)
        for (int i = 0; i < 2 * kBulkPlanes; ++i) mbar_inval(bar + i);
}

// y-FFT + Thomas forward elimination of one column block, sweeping k = 0..nz-1.
// Shared memory: kYZStages x [FFT buffer (mb padded sequences) | pivot chunk], then the
// Thomas state d'_{k-1} of every mode of the block.  Plane k+1 (spectrum and pivots)
// is copied with cp.async while plane k is transformed and eliminated.
// fp32: capped at 128 registers so that kYZResidentF32 CTAs fit on an SM (a few spilled
// bytes cost less than the lost residency)
template <typename T, bool W>
__global__ void __launch_bounds__(kYZThreads, sizeof(T) == 4 ? kYZResidentF32 : 1) k_yzfwd(Work w) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int g = find_grid(w.ystr_start, w.ngrids, blockIdx.x);
    const GridDev &G = w.grids[g];
    const int cb = blockIdx.x - __ldg(w.ystr_start + g);
    if constexpr (sizeof(T) == 4) {
        if (G.mb == 1 && !(W && G.wall_y)) {
            // whole-plane bulk copies need 16-byte aligned planes: even ny and spectrum offset
            if (((G.ny | (int)G.spec_off) & 1) == 0) yzfwd_bulk(w, G, cb, smem_raw);
            else yzfwd_pipe(w, G, cb, smem_raw);
            return;
        }
    }
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
// fp32: capped at 128 registers (no spill) so that kYZResidentF32 CTAs fit on an SM
template <typename T, bool W>
__global__ void __launch_bounds__(kYZThreads, sizeof(T) == 4 ? kYZResidentF32 : 1) k_yzbwd(Work w) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int g = find_grid(w.ystr_start, w.ngrids, blockIdx.x);
    const GridDev &G = w.grids[g];
    const int cb = blockIdx.x - __ldg(w.ystr_start + g);
    if constexpr (sizeof(T) == 4) {
        if (G.mb == 1 && !(W && G.wall_y)) {
            if (((G.ny | (int)G.spec_off) & 1) == 0) yzbwd_bulk(w, G, cb, smem_raw);
            else yzbwd_pipe(w, G, cb, smem_raw);
            return;
        }
    }
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
    // the (0,0) mode's solution (k_00) for slot 0 of block 0, loaded one plane ahead
    const bool own00 = cb == 0 && tid == 0;
    double s00n = own00 ? w.sol00[G.z_off + nz - 1] : 0.0;

    for (int k = nz - 1; k >= 0; --k) {
        const double s00 = s00n;
        if (own00 && k > 0) s00n = w.sol00[G.z_off + k - 1];
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
            if (cb == 0 && q == 0) ph = {(T)s00, (T)0};  // (0,0): k_00's solution
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

// ================================================================ k_yzslab
// Whole z extent of one column block resident in shared memory: load every plane,
// y-FFT of every plane, one tridiagonal solve per mode, inverse y-FFT, store.  The
// spectrum is read and written once (the streaming kernels read and write it twice).
// Shared memory: nz*mb padded FFT sequences, plane-major ([k][mm]); with cyclic
// reduction also three real arrays a, b, c of nz*nslot entries ([k][slot]).
//
// Tridiagonal algorithms (cr = G.cr_levels):
//   cr = 0: Thomas per mode with the plan's pivot table (as the streaming kernels);
//   cr = S: S levels of cyclic reduction (Hockney 1965; in place: at stride s the
//           equations i with (i+1) % 2s == 0 eliminate their neighbours i - s, i + s,
//           which are not written at that level), Thomas on the nz >> S remaining
//           equations of every mode, then S levels of back substitution.
// The (0,0) mode takes the fp64 solution of k_00.
template <typename T>
__device__ __forceinline__ T slab_lambda(const GridDev &G, int m, int n);
template <>
__device__ __forceinline__ float slab_lambda<float>(const GridDev &G, int m, int n) {
    const float sx = sinpif((float)m / (float)(G.wall_x ? 2 * G.nx : G.nx));
    const float sy = sinpif((float)n / (float)(G.wall_y ? 2 * G.ny : G.ny));
    return -4.f * (float)(G.rdx * G.rdx) * sx * sx - 4.f * (float)(G.rdy * G.rdy) * sy * sy;
}
template <>
__device__ __forceinline__ double slab_lambda<double>(const GridDev &G, int m, int n) {
    const double sx = sinpi((double)m / (G.wall_x ? 2 * G.nx : G.nx));
    const double sy = sinpi((double)n / (G.wall_y ? 2 * G.ny : G.ny));
    return -4.0 * G.rdx * G.rdx * sx * sx - 4.0 * G.rdy * G.rdy * sy * sy;
}

// fp32: capped at 128 registers, so that two CTAs fit on an SM where their slabs do
template <typename T, bool W>
__global__ void __launch_bounds__(kSlabThreads, sizeof(T) == 4 ? 2 : 1) k_yzslab(Work w) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int g = find_grid(w.slab_start, w.ngrids, blockIdx.x);
    const GridDev &G = w.grids[g];
    const int cb = blockIdx.x - __ldg(w.slab_start + g);
    const int ny = G.ny, nz = G.nz, mb = G.mb, ncb = G.ncb, nxh = G.nxh;
    const int N1 = G.ny1, N2 = G.ny2, sstride = fft_seq_len(N1, N2) + 1;
    const FDiv fN1 = G.fny1, fN2 = G.fny2, fmb = G.fmb;
    const int nslot = ny * mb;
    const int nvalid = min(mb, nxh - cb * mb);
    const int wall_y = W ? G.wall_y : 0;
    const cx<T> *twy = reinterpret_cast<const cx<T> *>(w.twy) + G.twy_off;
    const cx<T> *dcty = reinterpret_cast<const cx<T> *>(w.twy) + G.dcty_off;
    const int tid = threadIdx.x, nthr = blockDim.x;
    const int nseq = nz * mb;
    const size_t kst = (size_t)mb * sstride;  // distance between planes of one slot
    cx<T> *buf = reinterpret_cast<cx<T> *>(smem_raw);
    cx<T> *spec = reinterpret_cast<cx<T> *>(w.spec) + G.spec_off;
    const int total = nz * nslot;

    for (int t = tid; t < total; t += nthr) {
        const int k = t / nslot, q = t - k * nslot;
        const int j = (int)fdiv((unsigned)q, fmb), mm = q - j * mb;
        cx<T> v = {(T)0, (T)0};
        if (mm < nvalid) v = spec[((size_t)k * ncb + cb) * nslot + q];
        buf[k * kst + mm * sstride + pos_nat(wall_y ? dct_perm(j, ny) : j, fN2)] = v;
    }
    __syncthreads();
    fft_batch<T, -1>(buf, nseq, sstride, N1, N2, fN1, fN2, twy);
    if (wall_y) dct_post<T>(buf, nseq, sstride, ny, N1, N2, fN1, dcty);

    const T *az = zarr<T>(w.z.az, w.z.azf) + G.z_off;
    const T *cz = zarr<T>(w.z.cz, w.z.czf) + G.z_off;
    const double *s00 = w.sol00 + G.z_off;
    const int S = G.cr_levels;
    if (S == 0) {
        const T *tab = reinterpret_cast<const T *>(w.tab) + G.tab_off;
        for (int q = tid; q < nslot; q += nthr) {
            const int sn = (int)fdiv((unsigned)q, fmb), mm = q - sn * mb;
            cx<T> *col = buf + mm * sstride + pos_nat(sn, fN2);
            if (mm >= nvalid) continue;
            if (cb == 0 && q == 0) {
                for (int k = 0; k < nz; ++k) col[k * kst] = {(T)s00[k], (T)0};
                continue;
            }
            const T *tq = tab + (size_t)cb * nslot + q;
            const size_t tst = (size_t)ncb * nslot;
            cx<T> dp = {(T)0, (T)0};
#pragma unroll 4
            for (int k = 0; k < nz; ++k) {
                const T inv = tq[k * tst], a = az[k];
                const cx<T> r = col[k * kst];
                dp = {(r.x - a * dp.x) * inv, (r.y - a * dp.y) * inv};
                col[k * kst] = dp;
            }
            cx<T> ph = {(T)0, (T)0};
#pragma unroll 4
            for (int k = nz - 1; k >= 0; --k) {
                const T cp = cz[k] * tq[k * tst];
                const cx<T> d = col[k * kst];
                ph = {d.x - cp * ph.x, d.y - cp * ph.y};
                col[k * kst] = ph;
            }
        }
    } else {
        T *Ar = reinterpret_cast<T *>(smem_raw + (((size_t)nseq * sstride * sizeof(cx<T>) + 15) & ~(size_t)15));
        T *Br = Ar + total, *Cr = Br + total;
        // coefficients of every (level, slot); the singular and padding slots become identity rows
        for (int t = tid; t < total; t += nthr) {
            const int k = t / nslot, q = t - k * nslot;
            const int sn = (int)fdiv((unsigned)q, fmb), mm = q - sn * mb;
            const int m = cb * mb + mm, n = (sn / N2) + N1 * (sn - (sn / N2) * N2);
            cx<T> *e = buf + k * kst + mm * sstride + pos_nat(sn, fN2);
            if (mm >= nvalid || (cb == 0 && q == 0)) {
                Ar[t] = (T)0; Br[t] = (T)1; Cr[t] = (T)0;
                *e = {(mm < nvalid) ? (T)s00[k] : (T)0, (T)0};
            } else {
                const T a = az[k], c = cz[k];
                const T ez = (k == nz - 1) ? (T)G.ez_top : (T)0;  // Dirichlet outlet (0 otherwise)
                Ar[t] = a; Cr[t] = c; Br[t] = -(a + c) - ez + slab_lambda<T>(G, m, n);
            }
        }
        __syncthreads();
        auto D = [&](int k, int q) -> cx<T> & {
            const int sn = (int)fdiv((unsigned)q, fmb), mm = q - sn * mb;
            return buf[k * kst + mm * sstride + pos_nat(sn, fN2)];
        };
        for (int l = 0; l < S; ++l) {  // reduction: kept equations i = 2s(r+1) - 1
            const int s = 1 << l, s2 = s << 1, nk = nz / s2;
            for (int t = tid; t < nk * nslot; t += nthr) {
                const int r = t / nslot, q = t - r * nslot;
                const int i = s2 * (r + 1) - 1, im = i - s, ip = i + s;
                const int ti = i * nslot + q, tm = im * nslot + q, tp = ip * nslot + q;
                const T al = -Ar[ti] / Br[tm];
                cx<T> &di = D(i, q);
                const cx<T> dm = D(im, q);
                T na = al * Ar[tm], nb = Br[ti] + al * Cr[tm], nc = (T)0;
                cx<T> nd = {di.x + al * dm.x, di.y + al * dm.y};
                if (ip < nz) {
                    const T ga = -Cr[ti] / Br[tp];
                    const cx<T> dq = D(ip, q);
                    nc = ga * Cr[tp];
                    nb += ga * Ar[tp];
                    nd = {nd.x + ga * dq.x, nd.y + ga * dq.y};
                }
                Ar[ti] = na; Br[ti] = nb; Cr[ti] = nc;
                di = nd;
            }
            __syncthreads();
        }
        {   // Thomas on the reduced systems: equations 2^S (r+1) - 1, r < nz >> S
            const int st = 1 << S, R = nz >> S;
            for (int q = tid; q < nslot; q += nthr) {
                T cprev = (T)0;
                cx<T> dprev = {(T)0, (T)0};
                for (int r = 0; r < R; ++r) {
                    const int i = st * (r + 1) - 1, ti = i * nslot + q;
                    const T a = Ar[ti];
                    const T inv = (T)1 / (Br[ti] - a * cprev);
                    cx<T> &d = D(i, q);
                    dprev = {(d.x - a * dprev.x) * inv, (d.y - a * dprev.y) * inv};
                    cprev = Cr[ti] * inv;
                    Cr[ti] = cprev;
                    d = dprev;
                }
                cx<T> x = {(T)0, (T)0};
                for (int r = R - 1; r >= 0; --r) {
                    const int i = st * (r + 1) - 1;
                    cx<T> &d = D(i, q);
                    const T c = Cr[i * nslot + q];
                    x = {d.x - c * x.x, d.y - c * x.y};
                    d = x;
                }
            }
            __syncthreads();
        }
        for (int l = S - 1; l >= 0; --l) {  // back substitution of the equations eliminated at level l
            const int s = 1 << l, cnt = (nz / s + 1) >> 1;
            for (int t = tid; t < cnt * nslot; t += nthr) {
                const int r = t / nslot, q = t - r * nslot;
                const int i = s * (2 * r + 1) - 1;
                if (i >= nz) continue;
                const int ti = i * nslot + q;
                cx<T> &d = D(i, q);
                cx<T> v = d;
                if (i - s >= 0) {
                    const cx<T> xm = D(i - s, q);
                    v = {v.x - Ar[ti] * xm.x, v.y - Ar[ti] * xm.y};
                }
                if (i + s < nz) {
                    const cx<T> xp = D(i + s, q);
                    v = {v.x - Cr[ti] * xp.x, v.y - Cr[ti] * xp.y};
                }
                const T inv = (T)1 / Br[ti];
                d = {v.x * inv, v.y * inv};
            }
            __syncthreads();
        }
    }
    __syncthreads();
    if (wall_y) dct_pre<T>(buf, nseq, sstride, ny, N1, N2, fN1, dcty);
    fft_batch<T, +1>(buf, nseq, sstride, N1, N2, fN1, fN2, twy);
    for (int t = tid; t < total; t += nthr) {
        const int k = t / nslot, q = t - k * nslot;
        const int j = (int)fdiv((unsigned)q, fmb), mm = q - j * mb;
        if (mm < nvalid)
            spec[((size_t)k * ncb + cb) * nslot + q] = buf[k * kst + mm * sstride + pos_nat(wall_y ? dct_perm(j, ny) : j, fN2)];
    }
}

// ================================================================ split y/z path
// y transform of one (plane, column block): the spectrum chunk of ny*mb x-modes is
// loaded, transformed along y (FFT, or DCT-II / DCT-III input stage in a wall-bounded
// y) and written back in place, in slot order (forward) or row order (inverse).
// Every (plane, block) is independent, so the launch has nz*ncb blocks per grid.
template <typename T, int DIR, bool W>
__global__ void __launch_bounds__(kYZThreads, sizeof(T) == 4 ? 4 : 1) k_yfft(Work w) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int g = find_grid(w.yfft_start, w.ngrids, blockIdx.x);
    const GridDev &G = w.grids[g];
    const int lb = blockIdx.x - __ldg(w.yfft_start + g);
    const int ncb = G.ncb, k = lb / ncb, cb = lb - k * ncb;
    const int ny = G.ny, mb = G.mb, nxh = G.nxh;
    const int N1 = G.ny1, N2 = G.ny2, sstride = fft_seq_len(N1, N2) + 1;
    const FDiv fN1 = G.fny1, fN2 = G.fny2, fmb = G.fmb;
    const int nslot = ny * mb;
    const int nvalid = min(mb, nxh - cb * mb);
    const int wall_y = W ? G.wall_y : 0;
    const cx<T> *twy = reinterpret_cast<const cx<T> *>(w.twy) + G.twy_off;
    const cx<T> *dcty = reinterpret_cast<const cx<T> *>(w.twy) + G.dcty_off;
    cx<T> *buf = reinterpret_cast<cx<T> *>(smem_raw);
    cx<T> *pl = reinterpret_cast<cx<T> *>(w.spec) + G.spec_off + ((size_t)k * ncb + cb) * nslot;
    const int tid = threadIdx.x, nthr = blockDim.x;
    for (int t = tid; t < nslot; t += nthr) {
        const int r = (int)fdiv((unsigned)t, fmb), mm = t - r * mb;
        // forward: row r of the x-spectrum; inverse: slot r (FFT output order)
        const int pos = DIR < 0 ? pos_nat(wall_y ? dct_perm(r, ny) : r, fN2) : pos_nat(r, fN2);
        buf[mm * sstride + pos] = (mm < nvalid) ? pl[t] : cx<T>{(T)0, (T)0};
    }
    __syncthreads();
    if (DIR > 0 && wall_y) dct_pre<T>(buf, mb, sstride, ny, N1, N2, fN1, dcty);
    fft_batch<T, DIR>(buf, mb, sstride, N1, N2, fN1, fN2, twy);
    if (DIR < 0 && wall_y) dct_post<T>(buf, mb, sstride, ny, N1, N2, fN1, dcty);
    for (int t = tid; t < nslot; t += nthr) {
        const int r = (int)fdiv((unsigned)t, fmb), mm = t - r * mb;
        const int pos = DIR < 0 ? pos_nat(r, fN2) : pos_nat(wall_y ? dct_perm(r, ny) : r, fN2);
        if (mm < nvalid) pl[t] = buf[mm * sstride + pos];
    }
}

// Thomas sweeps of the split path: one thread per mode of a grid (slot gs of the
// flattened [column block][slot] index, so plane k of the spectrum is one contiguous
// run of ncb*nslot modes), pivots from the plan's table.  Forward overwrites the
// spectrum with d'; the (0,0) mode passes through (k_00 solves it); backward turns
// d' into phi_hat.
template <typename T, bool BWD>
__global__ void __launch_bounds__(kSweepThreads) k_zsweep(Work w) {
    const int g = find_grid(w.sweep_start, w.ngrids, blockIdx.x);
    const GridDev &G = w.grids[g];
    const int gs = (blockIdx.x - __ldg(w.sweep_start + g)) * kSweepThreads + threadIdx.x;
    const int nslot = G.ny * G.mb, M = G.ncb * nslot, nz = G.nz;
    if (gs >= M) return;
    const int cb = gs / nslot, q = gs - cb * nslot;
    const int mm = q - (int)fdiv((unsigned)q, G.fmb) * G.mb;
    if (cb * G.mb + mm >= G.nxh) return;  // padding column of the last block
    const bool singular = gs == 0;
    cx<T> *sp = reinterpret_cast<cx<T> *>(w.spec) + G.spec_off + gs;
    const T *tb = reinterpret_cast<const T *>(w.tab) + G.tab_off + gs;
    const T *a = zarr<T>(w.z.az, w.z.azf) + G.z_off;
    const T *c = zarr<T>(w.z.cz, w.z.czf) + G.z_off;
    cx<T> s = {(T)0, (T)0};
    if (!BWD) {
#pragma unroll 8
        for (int k = 0; k < nz; ++k) {
            const cx<T> r = sp[(size_t)k * M];
            const T inv = tb[(size_t)k * M], ak = a[k];
            s = singular ? r : cx<T>{(r.x - ak * s.x) * inv, (r.y - ak * s.y) * inv};
            sp[(size_t)k * M] = s;
        }
    } else {
#pragma unroll 8
        for (int k = nz - 1; k >= 0; --k) {
            const cx<T> d = sp[(size_t)k * M];
            const T cp = c[k] * tb[(size_t)k * M];
            s = singular ? d : cx<T>{d.x - cp * s.x, d.y - cp * s.y};
            sp[(size_t)k * M] = s;
        }
    }
}

// ================================================================ k_plane_sums
// The plane sums of the right-hand side (and, in a refinement pass, of phi) for k_00:
// the forward x kernels leave one slot per row block (two with the half-block CTAs); one
// warp per plane adds its slots, lane-strided then by a butterfly of shuffles (a fixed
// order), and stores the sum in the plane's first slot, the only one k_00 reads.  Spread
// over many SMs, since the fp64 pipe of one SM would take the whole sum tens of
// microseconds.
constexpr int kPlaneSumThreads = 256;
__global__ void __launch_bounds__(kPlaneSumThreads) k_plane_sums(Work w, int first_solve) {
    const GridDev &G = w.grids[blockIdx.y];
    const int k = blockIdx.x * (kPlaneSumThreads / 32) + (threadIdx.x >> 5), lane = threadIdx.x & 31;
    if (k >= G.nz) return;  // warp-uniform
    const int np = G.nrb * (w.xfwd_split ? 2 : 1);
    double *pk = w.partial + G.part_off + (size_t)k * np, *qk = w.partial_phi + G.part_off + (size_t)k * np;
    double S = 0.0, P = 0.0;
    for (int r = lane; r < np; r += 32) {
        S += pk[r];
        if (!first_solve) P += qk[r];
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        S += __shfl_xor_sync(0xffffffffu, S, o);
        if (!first_solve) P += __shfl_xor_sync(0xffffffffu, P, o);
    }
    // every lane's loads are done (the shuffles consumed them) and only lane 0 read slot 0
    if (lane == 0) {
        pk[0] = S;
        if (!first_solve) qk[0] = P;
    }
}

// In-place inclusive prefix sums of a[0..n) in fp64 (rev: suffix sums, a[i] = sum over
// j >= i), all threads of the block: each thread scans a contiguous chunk, the chunk totals
// are scanned by warp shuffles and across warps through wsum[blockDim / 32]; a fixed order.
__device__ void block_scan_fp64(double *a, int n, bool rev, double *wsum) {
    const int T = blockDim.x, t = threadIdx.x, lane = t & 31, wid = t >> 5, nw = T >> 5;
    const int per = (n + T - 1) / T, b0 = min(n, t * per), b1 = min(n, b0 + per);
    auto at = [&](int i) -> double & { return a[rev ? n - 1 - i : i]; };
    double loc = 0.0;
    for (int i = b0; i < b1; ++i) {
        loc += at(i);
        at(i) = loc;
    }
    double x = loc;  // inclusive scan of the chunk totals within the warp
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const double y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    double ex = __shfl_up_sync(0xffffffffu, x, 1);  // exclusive: the chunks before this one
    if (lane == 0) ex = 0.0;
    if (lane == 31) wsum[wid] = x;
    __syncthreads();
    if (wid == 0) {
        double v = lane < nw ? wsum[lane] : 0.0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const double y = __shfl_up_sync(0xffffffffu, v, o);
            if (lane >= o) v += y;
        }
        if (lane < nw) wsum[lane] = v;
    }
    __syncthreads();
    const double off = wid > 0 ? ex + wsum[wid - 1] : ex;
    for (int i = b0; i < b1; ++i) at(i) += off;
    __syncthreads();
}

// ================================================================ k_00 (fp64, one CTA per grid)
template <typename T>
__global__ void __launch_bounds__(256) k_00(Work w, int first_solve) {
    // Shared memory: right-hand side, hz, the flux terms hz_k d_k, their running sums,
    // the increments of phi, phi, and the plane means of the phi being refined; every
    // array has nz+1 entries (the plan reserves ten).
    extern __shared__ double sh00[];
    __shared__ double red[8];
    const int g = blockIdx.x;
    const GridDev &G = w.grids[g];
    const int nz = G.nz, nrb = G.nrb, zo = G.z_off;
    const int L = nz + 1;
    double *rhs = sh00, *hz = sh00 + L;
    double *A0 = sh00 + 2 * L, *B0 = A0 + L, *C0 = B0 + L, *D0 = C0 + L;
    double *A1 = D0 + L;
    const double *part = w.partial + G.part_off, *partp = w.partial_phi + G.part_off;
    double *Pk = A1;  // plane means of the phi being refined
    double loc = 0.0, locp = 0.0;
    bool bad = false;
    // plane sums: k_plane_sums left each plane's in its first slot
    const int np = nrb * (w.xfwd_split ? 2 : 1);
    double lmax = 0.0;
    for (int k = threadIdx.x; k < nz; k += blockDim.x) {
        const double m = part[(size_t)k * np] * G.inv_nxy;  // plane mean of b (first solve) or of the residual
        if (!isfinite(m)) bad = true;
        const double h = w.z.hz[zo + k];
        rhs[k] = m;
        hz[k] = h;
        lmax = fmax(lmax, fabs(m));
        if (!first_solve) {
            Pk[k] = partp[(size_t)k * np] * G.inv_nxy;
            locp += h * Pk[k];
        }
    }
    if (bad) atomicOr(w.err, 1u << 6);  // IBF_ERR_NONFINITE
    __syncthreads();
    // In a refinement pass rhs[k] is already the plane mean of the residual
    // b - <b> - L phi (summed from its per-cell values, which are small once phi is
    // close): forming it instead from the plane means of b and of phi would carry the
    // rounding of phi's plane means, amplified by the z part of L (up to 1/(hz gz) next
    // to a stretched wall), into the correction.
    for (int k = threadIdx.x; k < nz; k += blockDim.x) loc += hz[k] * rhs[k];
    const double tot = Red<F64Arith>::sum(loc, red);
    // weighted mean of the phi being refined: the correction also removes it, so that
    // phi + delta keeps a zero weighted mean (L cannot see a constant)
    const double totp = first_solve ? 0.0 : Red<F64Arith>::sum(locp, red);
    // a Dirichlet outlet makes the (0,0) system regular: nothing to remove
    if (threadIdx.x == 0) red[0] = G.dir_top ? 0.0 : tot / G.sum_hz;
    __syncthreads();
    const double mean = red[0];
    if (first_solve) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) lmax = fmax(lmax, __shfl_xor_sync(0xffffffffu, lmax, o));
        __syncthreads();  // red[0] (the mean) has been read by every thread
        if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = lmax;
        __syncthreads();
        if (threadIdx.x == 0) {
            w.mean_b[g] = mean;
            double scale = 0.0;
            for (int i = 0; i < (int)(blockDim.x >> 5); ++i) scale = fmax(scale, red[i]);
            // compatibility defect large compared with the plane means -> warning
            if (fabs(mean) > 1e-8 * scale && fabs(mean) > 0.0) atomicOr(w.err, 1u << 7);
        }
        __syncthreads();
    }
    // The (0,0) system in flux form.  Row k of L along z, times hz_k, is a difference of
    // face fluxes, hz_k (L phi)_k = F_{k+1/2} - F_{k-1/2} with F_{k+1/2} =
    // (phi_{k+1} - phi_k) / gz_{k+1} and F_{-1/2} = 0 at the bottom wall, so
    //   F_{k+1/2} = S_k = sum_{j <= k} hz_j d_j,      d = right-hand side less its mean,
    //   phi_k     = phi_{k+1} - gz_{k+1} S_k          (integrated down from level nz-1).
    // Neumann top: the top flux is zero (S_{nz-1} = 0 up to rounding, since d has zero
    // weighted mean), phi_{nz-1} is pinned to 0 and the weighted mean removed below.
    // Dirichlet outlet: the top flux is -hz_{nz-1} ez_top phi_{nz-1} = S_{nz-1}, which
    // fixes phi_{nz-1}.  The two running sums are the exact solve of the system; unlike
    // an elimination on the rows a_k, -(a_k + c_k), c_k (whose reduced diagonals cancel
    // by orders of magnitude on a stretched grid) they leave a residual at the rounding
    // of the fluxes.  The running sums are block-wide scans (a fixed order), the
    // divisions by 1/gz are parallel.
    double *S = A0, *inc = C0;
    for (int k = threadIdx.x; k < nz; k += blockDim.x) A0[k] = hz[k] * (rhs[k] - mean);
    __syncthreads();
    block_scan_fp64(S, nz, false, red);  // S_k, in place
    for (int k = threadIdx.x; k + 1 < nz; k += blockDim.x) inc[k] = S[k] / w.z.rgzf[zo + k + 1];
    __syncthreads();
    block_scan_fp64(inc, nz - 1, true, red);  // inc[k] = sum_{j = k}^{nz-2} gz_{j+1} S_j
    const double ph_top = G.dir_top ? -S[nz - 1] / (hz[nz - 1] * G.ez_top) : 0.0;
    for (int k = threadIdx.x; k < nz; k += blockDim.x) D0[k] = k + 1 < nz ? ph_top - inc[k] : ph_top;
    __syncthreads();
    double lsv = 0.0;
    for (int k = threadIdx.x; k < nz; k += blockDim.x) {
        const double ph = D0[k];
        rhs[k] = ph;
        lsv += hz[k] * ph;
    }
    __syncthreads();
    const double sv = Red<F64Arith>::sum(lsv, red);
    if (threadIdx.x == 0) rhs[nz] = G.dir_top ? 0.0 : (sv + totp) / G.sum_hz;  // weighted mean to remove
    __syncthreads();
    const double mphi = rhs[nz];
    cx<T> *spec = reinterpret_cast<cx<T> *>(w.spec) + G.spec_off;
    const size_t stride = (size_t)G.ncb * G.ny * G.mb;
    for (int k = threadIdx.x; k < nz; k += blockDim.x) {
        const double v = rhs[k] - mphi;
        // split and spectral-z paths: slot (0,0) of the y-transformed spectrum; the
        // streaming backward kernel and the slab kernel read sol00
        if (G.yzk >= 2) spec[(size_t)k * stride] = {(T)v, (T)0};
        w.sol00[zo + k] = v;
    }
}

// ================================================================ spectral z
// yz_kernel 4, uniform z with Neumann walls at both ends: the cell-centred second
// difference along z is then diagonalised by the DCT-II (eigenvalues
// -(4/hz^2) sin^2(pi l / (2 nz)), l < nz), so after the y transforms of the split path
// every mode (m, n, l) is divided by lambda_x(m) + lambda_y(n) + lambda_z(l) and no
// tridiagonal sweep remains.  The same slot of every plane's spectrum is one z line;
// a CTA takes zdct_lines<T>() consecutive slots: DCT-II along z (Makhoul reorder, FFT,
// post-twiddle), division, DCT-III (pre-twiddle, inverse FFT, un-reordering; the unscaled
// pair returns nz times the input, folded into the division).  The (0,0) column is
// overwritten afterwards by k_00 (fp64, compatibility and mean handling).
template <typename T> __host__ __device__ constexpr int zdct_lines() { return sizeof(T) == 4 ? kZdctLinesF32 : kZdctLinesF64; }
template <typename T> __device__ __forceinline__ T sinpi_T(T x);
template <> __device__ __forceinline__ float sinpi_T<float>(float x) { return sinpif(x); }
template <> __device__ __forceinline__ double sinpi_T<double>(double x) { return sinpi(x); }

template <typename T>
__global__ void __launch_bounds__(kYZThreads, sizeof(T) == 4 ? 4 : 1) k_zdct(Work w) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    constexpr int TM = zdct_lines<T>();
    const int g = find_grid(w.zdct_start, w.ngrids, blockIdx.x);
    const GridDev &G = w.grids[g];
    const int ny = G.ny, nz = G.nz, mb = G.mb;
    const long long M = (long long)G.ncb * ny * mb;  // slots per plane
    const long long s0 = (long long)(blockIdx.x - __ldg(w.zdct_start + g)) * TM;
    const int N1 = G.nz1, N2 = G.nz2, sstride = fft_seq_len(N1, N2) + 1;
    const FDiv fN1 = G.fnz1, fN2 = G.fnz2;
    const cx<T> *twz = reinterpret_cast<const cx<T> *>(w.twy) + G.twz_off;
    const cx<T> *dctz = reinterpret_cast<const cx<T> *>(w.twy) + G.dctz_off;
    cx<T> *buf = reinterpret_cast<cx<T> *>(smem_raw);
    cx<T> *spec = reinterpret_cast<cx<T> *>(w.spec) + G.spec_off;
    const int tid = threadIdx.x, nthr = blockDim.x;
    for (int t = tid; t < TM * nz; t += nthr) {  // plane k, line i: consecutive threads on consecutive slots
        const int k = t / TM, i = t - k * TM;
        const long long s = s0 + i;
        buf[i * sstride + pos_nat(dct_perm(k, nz), fN2)] = s < M ? spec[(size_t)k * M + s] : cx<T>{(T)0, (T)0};
    }
    __syncthreads();
    fft_batch<T, -1>(buf, TM, sstride, N1, N2, fN1, fN2, twz);
    dct_post<T>(buf, TM, sstride, nz, N1, N2, fN1, dctz);
    const T cx_ = (T)(4.0 * G.rdx * G.rdx), cy_ = (T)(4.0 * G.rdy * G.rdy);
    const T cz_ = (T)(4.0 * nz * nz / (G.sum_hz * G.sum_hz));
    const T dxn = (T)(G.wall_x ? 2 * G.nx : G.nx), dyn = (T)(G.wall_y ? 2 * ny : ny);
    for (int t = tid; t < TM * nz; t += nthr) {
        const int i = t / nz, l = t - i * nz;
        const long long s = s0 + i;
        cx<T> &v = buf[i * sstride + pos_tr(l, N1, N2, fN1)];
        T f = (T)0;
        if (s < M) {
            const int mm = (int)(s % mb);
            const long long rest = s / mb;
            const int j = (int)(rest % ny), cb = (int)(rest / ny);
            const int m = cb * mb + mm, n = (j / G.ny2) + G.ny1 * (j % G.ny2);  // slot row j holds y-mode n
            if (m < G.nxh) {
                const T sx = sinpi_T<T>((T)m / dxn), sy = sinpi_T<T>((T)n / dyn),
                        sz = sinpi_T<T>((T)l / (T)(2 * nz));
                const T lam = -(cx_ * sx * sx + cy_ * sy * sy + cz_ * sz * sz);
                if (lam != (T)0) f = (T)1 / (lam * (T)nz);
            }
        }
        v = {v.x * f, v.y * f};
    }
    __syncthreads();
    dct_pre<T>(buf, TM, sstride, nz, N1, N2, fN1, dctz);
    fft_batch<T, +1>(buf, TM, sstride, N1, N2, fN1, fN2, twz);
    for (int t = tid; t < TM * nz; t += nthr) {
        const int k = t / TM, i = t - k * TM;
        const long long s = s0 + i;
        if (s < M) spec[(size_t)k * M + s] = buf[i * sstride + pos_nat(dct_perm(k, nz), fN2)];
    }
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
                const double ez = (k == nz - 1) ? G.ez_top : 0.0;  // Dirichlet outlet (0 otherwise)
                inv = 1.0 / (-(az[k] + cz[k]) - ez + lam - az[k] * cp);
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
    const int wpb = kPlaneSumThreads / 32;
    k_plane_sums<<<dim3((unsigned)((maxnz + wpb - 1) / wpb), (unsigned)w.ngrids), kPlaneSumThreads, 0, st>>>(w, first_solve);
    if (mixed) k_00<float><<<w.ngrids, 256, smem, st>>>(w, first_solve);
    else k_00<double><<<w.ngrids, 256, smem, st>>>(w, first_solve);
    return cudaGetLastError();
}

cudaError_t launch_yzslab(int mixed, const Work &w, int nblk, size_t smem, cudaStream_t st) {
    if (nblk <= 0) return cudaSuccess;
    if (mixed) {
        if (w.walls) k_yzslab<float, true><<<grid1(nblk), kSlabThreads, smem, st>>>(w);
        else k_yzslab<float, false><<<grid1(nblk), kSlabThreads, smem, st>>>(w);
    } else {
        if (w.walls) k_yzslab<double, true><<<grid1(nblk), kSlabThreads, smem, st>>>(w);
        else k_yzslab<double, false><<<grid1(nblk), kSlabThreads, smem, st>>>(w);
    }
    return cudaGetLastError();
}

cudaError_t launch_yfft(int mixed, int inverse, const Work &w, int nblk, size_t smem, cudaStream_t st) {
    if (nblk <= 0) return cudaSuccess;
    const dim3 gr = grid1(nblk);
    if (mixed) {
        if (inverse) {
            if (w.walls) k_yfft<float, 1, true><<<gr, kYZThreads, smem, st>>>(w);
            else k_yfft<float, 1, false><<<gr, kYZThreads, smem, st>>>(w);
        } else {
            if (w.walls) k_yfft<float, -1, true><<<gr, kYZThreads, smem, st>>>(w);
            else k_yfft<float, -1, false><<<gr, kYZThreads, smem, st>>>(w);
        }
    } else {
        if (inverse) {
            if (w.walls) k_yfft<double, 1, true><<<gr, kYZThreads, smem, st>>>(w);
            else k_yfft<double, 1, false><<<gr, kYZThreads, smem, st>>>(w);
        } else {
            if (w.walls) k_yfft<double, -1, true><<<gr, kYZThreads, smem, st>>>(w);
            else k_yfft<double, -1, false><<<gr, kYZThreads, smem, st>>>(w);
        }
    }
    return cudaGetLastError();
}

cudaError_t launch_zsweep(int mixed, int backward, const Work &w, int nblk, cudaStream_t st) {
    if (nblk <= 0) return cudaSuccess;
    const dim3 gr = grid1(nblk);
    if (mixed) {
        if (backward) k_zsweep<float, true><<<gr, kSweepThreads, 0, st>>>(w);
        else k_zsweep<float, false><<<gr, kSweepThreads, 0, st>>>(w);
    } else {
        if (backward) k_zsweep<double, true><<<gr, kSweepThreads, 0, st>>>(w);
        else k_zsweep<double, false><<<gr, kSweepThreads, 0, st>>>(w);
    }
    return cudaGetLastError();
}

cudaError_t launch_build_table(int mixed, const Work &w, int nblk, cudaStream_t st) {
    if (mixed) k_build_table<float><<<grid1(nblk), 256, 0, st>>>(w);
    else k_build_table<double><<<grid1(nblk), 256, 0, st>>>(w);
    return cudaGetLastError();
}

cudaError_t launch_zdct(int mixed, const Work &w, int nblk, size_t smem, cudaStream_t st) {
    if (nblk <= 0) return cudaSuccess;
    if (mixed) k_zdct<float><<<grid1(nblk), kYZThreads, smem, st>>>(w);
    else k_zdct<double><<<grid1(nblk), kYZThreads, smem, st>>>(w);
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
            set((const void *)k_yzslab<float, W>);
            set((const void *)k_yfft<float, -1, W>);
            set((const void *)k_yfft<float, 1, W>);
        } else {
            set((const void *)k_yzfwd<double, W>);
            set((const void *)k_yzbwd<double, W>);
            set((const void *)k_yzslab<double, W>);
            set((const void *)k_yfft<double, -1, W>);
            set((const void *)k_yfft<double, 1, W>);
        }
    };
    set_all(std::false_type{});
    set_all(std::true_type{});
    if (mixed) set((const void *)k_00<float>);
    else set((const void *)k_00<double>);
    if (mixed) set((const void *)k_zdct<float>);
    else set((const void *)k_zdct<double>);
    return e;
}

}  // namespace ibf

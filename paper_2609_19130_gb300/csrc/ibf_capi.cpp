// ibf_capi.cpp -- host side of libibf: plan construction (validation, grid
// geometry, tridiagonal coefficients, twiddles, pivot tables, launch shapes,
// workspace) and the C ABI declared in include/ibf.h.
#include "../../include/ibf.h"

#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <new>
#include <string>
#include <vector>

#include "ibf_internal.h"
#include "ibf_viscous.h"

using namespace ibf;

namespace {

thread_local std::string g_last_error;

ibf_status cuda_fail(cudaError_t e, const char *what) {
    g_last_error = std::string(what) + ": " + cudaGetErrorString(e);
    (void)cudaGetLastError();  // do not leave a non-sticky error pending for the caller's next CUDA call
    return IBF_ERR_CUDA;
}

const int kFftSizes[] = {1, 2, 3, 4, 6, 8, 12, 16, 24, 32};

bool in_sizes(int n) {
    for (int s : kFftSizes)
        if (s == n) return true;
    return false;
}

// n = n1 * n2 with both factors register-DFT sizes, n1 >= n2, as balanced as possible.
bool factor(int n, int *n1, int *n2) {
    int best1 = -1, best2 = -1;
    for (int a : kFftSizes) {
        if (n % a) continue;
        const int b = n / a;
        if (!in_sizes(b) || a < b) continue;
        if (best1 < 0 || a < best1) { best1 = a; best2 = b; }
    }
    if (best1 < 0) return false;
    *n1 = best1;
    *n2 = best2;
    return true;
}

struct GridHost {
    ibf_grid g;
    std::vector<double> zf;
    GridDev d;
    ibf_tuning tun;  // resolved launch shape
};

struct ProfRec {
    const char *name;
    cudaEvent_t e0, e1;
};

}  // namespace

struct ibf_plan {
    int device = 0;
    int ngrids = 0;
    ibf_opts opts{};
    int mixed = 0;
    std::vector<GridHost> grids;
    std::vector<void *> allocs;
    Work work{};
    size_t xsmem = 0, yzsmem = 0, slabsmem = 0, yfftsmem = 0, zdctsmem = 0;
    int nzdctblk = 0;
    // viscous solve: pivots of (I - beta Lz) per grid (6 (nz+1) entries at 6 z_off) and the
    // shared memory of its y kernel
    double *helm = nullptr, *fxy = nullptr;
    float *helmf = nullptr, *fxyf = nullptr;
    long long *fxy_off_dev = nullptr;   // per grid: offset of its x / y factors (nxh + ny entries)
    std::vector<long long> fxy_off;
    size_t helmsmem = 0, smemcap = 0;
    bool helm_valid = false;            // the tables hold the factors of helm_beta
    double helm_beta = 0.0;
    int nxblk = 0, nyzblk = 0, nstrblk = 0, nslabblk = 0, nyfftblk = 0, nsweepblk = 0, maxnz = 0;
    long long ws_bytes = 0;
    long long total_cells = 0;
    cudaStream_t last_stream = nullptr;
    // profiling
    bool prof = false;
    std::vector<ProfRec> prof_pending;
    std::vector<cudaEvent_t> ev_pool;
    std::vector<std::pair<const char *, std::pair<long long, double>>> prof_acc;
};

namespace {

// Test hook: IBF_FAULT_OOM_AT=n makes the n-th plan allocation of the process fail
// (one counter for every allocation, whatever its element type).
bool inject_alloc_failure() {
    static std::mutex mu;
    static int countdown = -2;
    std::lock_guard<std::mutex> lk(mu);
    if (countdown == -2) {
        const char *f = getenv("IBF_FAULT_OOM_AT");
        countdown = f ? atoi(f) : -1;
    }
    return countdown > 0 && --countdown == 0;
}

template <typename P> ibf_status dalloc(ibf_plan *pl, P **out, size_t bytes) {
    *out = nullptr;
    if (bytes == 0) bytes = 16;
    if (inject_alloc_failure()) {
        g_last_error = "injected allocation failure";
        return IBF_ERR_OOM;
    }
    void *p = nullptr;
    cudaError_t e = cudaMalloc(&p, bytes);
    if (e != cudaSuccess) {
        (void)cudaGetLastError();
        g_last_error = std::string("cudaMalloc: ") + cudaGetErrorString(e);
        return IBF_ERR_OOM;
    }
    pl->allocs.push_back(p);
    pl->ws_bytes += (long long)bytes;
    *out = static_cast<P *>(p);
    return IBF_OK;
}

void free_all(ibf_plan *pl) {
    for (void *p : pl->allocs) cudaFree(p);
    pl->allocs.clear();
    for (auto &r : pl->prof_pending) { cudaEventDestroy(r.e0); cudaEventDestroy(r.e1); }
    pl->prof_pending.clear();
    for (auto e : pl->ev_pool) cudaEventDestroy(e);
    pl->ev_pool.clear();
}

}  // namespace

// Host validation of one grid descriptor; fills zf with the nz + 1 z faces (the
// caller's, or the tanh map).  Shared by ibf_projection_plan and ibf_project_noalloc.
ibf_status ibf::validate_grid(const ibf_grid *g, std::vector<double> &zf) {
    if (g->nx < 1 || g->ny < 1 || g->nz < 1) return IBF_ERR_INVALID_ARG;
    if (!(g->lx > 0) || !(g->ly > 0) || !(g->lz > 0)) return IBF_ERR_INVALID_ARG;
    if (!std::isfinite(g->lx) || !std::isfinite(g->ly) || !std::isfinite(g->lz)) return IBF_ERR_INVALID_ARG;
    if ((long long)g->nx * g->ny * g->nz > (1ll << 34)) return IBF_ERR_UNSUPPORTED_SIZE;
    const int bcs[4] = {g->bc_x, g->bc_y, g->bc_zlo, g->bc_zhi};
    for (int b : bcs)
        if (b < IBF_BC_PERIODIC || b > IBF_BC_DIRICHLET) return IBF_ERR_INVALID_ARG;
    if (g->bc_x == IBF_BC_DIRICHLET || g->bc_y == IBF_BC_DIRICHLET) return IBF_ERR_UNSUPPORTED_BC;
    if (g->bc_zlo != IBF_BC_NEUMANN || g->bc_zhi == IBF_BC_PERIODIC) return IBF_ERR_UNSUPPORTED_BC;
    int a, b;
    if (!factor(g->nx, &a, &b) || !factor(g->ny, &a, &b)) return IBF_ERR_UNSUPPORTED_SIZE;
    const int nz = g->nz;
    zf.assign(nz + 1, 0.0);
    if (g->zf) {
        for (int k = 0; k <= nz; ++k) {
            zf[k] = g->zf[k];
            if (!std::isfinite(zf[k])) return IBF_ERR_INVALID_ARG;
        }
        if (std::fabs(zf[0]) > 1e-12 * g->lz || std::fabs(zf[nz] - g->lz) > 1e-12 * g->lz) return IBF_ERR_INVALID_ARG;
        for (int k = 0; k < nz; ++k)
            if (!(zf[k + 1] > zf[k])) return IBF_ERR_INVALID_ARG;
    } else {
        if (!std::isfinite(g->beta) || g->beta < 0) return IBF_ERR_INVALID_ARG;
        for (int k = 0; k <= nz; ++k)
            zf[k] = (g->beta == 0.0) ? g->lz * (double)k / nz
                                     : 0.5 * g->lz * (1.0 + std::tanh(g->beta * (2.0 * k / nz - 1.0)) / std::tanh(g->beta));
        for (int k = 0; k < nz; ++k)
            if (!(zf[k + 1] > zf[k])) return IBF_ERR_INVALID_ARG;  // beta so large that faces collapse
    }
    zf[0] = 0.0;
    zf[nz] = g->lz;
    return IBF_OK;
}

namespace {

// magic numbers of FDiv (round-up method, valid for dividends below 2^31)
FDiv make_fdiv(unsigned d) {
    FDiv f;
    f.d = d;
    unsigned s = 0;
    while ((1ull << s) < d) ++s;
    f.s = s;
    f.m = (unsigned)((((1ull << 32) * ((1ull << s) - d)) / d) + 1);
    return f;
}

// exp(-2 pi i r / n), r < n, in fp64 (host libm)
// Four-step twiddles w^(a b), w = exp(-2 pi i / n), of an n = n1 n2 FFT, in the two
// layouts their passes read with consecutive lanes on consecutive entries: forward
// F[q n2 + c] = w^(q c) (q < n1, c < n2; the column pass, lanes over columns c), then
// inverse I[p n1 + q1] = w^(p q1) (p < n2, q1 < n1; the row pass, lanes over rows q1).
void twiddles(int n, int n1, std::vector<double> &out) {
    const int n2 = n / n1;
    out.resize(4 * (size_t)n);
    auto put = [&](size_t i, long long e) {
        const double a = 2.0 * M_PI * (double)(e % n) / (double)n;
        out[2 * i] = std::cos(a);
        out[2 * i + 1] = -std::sin(a);
    };
    for (int q = 0; q < n1; ++q)
        for (int c = 0; c < n2; ++c) put((size_t)q * n2 + c, (long long)q * c);
    for (int p = 0; p < n2; ++p)
        for (int q1 = 0; q1 < n1; ++q1) put((size_t)n + (size_t)p * n1 + q1, (long long)p * q1);
}

// exp(-i pi m / (2n)), m < n: the DCT-II post-twiddles (Makhoul)
void dct_twiddles(int n, std::vector<double> &out) {
    out.resize(2 * (size_t)n);
    for (int m = 0; m < n; ++m) {
        const double a = M_PI * (double)m / (2.0 * (double)n);
        out[2 * m] = std::cos(a);
        out[2 * m + 1] = -std::sin(a);
    }
}

// x-modes kept by the x transform: nx/2 + 1 (real FFT) or nx (DCT-II, wall-bounded x)
int x_modes(const ibf_grid &g) { return g.bc_x == IBF_BC_NEUMANN ? g.nx : g.nx / 2 + 1; }

ibf_status upload(const void *host, void *dev, size_t bytes) {
    cudaError_t e = cudaMemcpy(dev, host, bytes, cudaMemcpyHostToDevice);
    return e == cudaSuccess ? IBF_OK : cuda_fail(e, "cudaMemcpy");
}

#define IBF_TRY(x) do { ibf_status _s = (x); if (_s != IBF_OK) return _s; } while (0)

// dynamic shared memory a kernel may request (the opt-in maximum less a margin for the
// kernels' static shared memory)
size_t smem_cap(const cudaDeviceProp &prop) { return smem_cap_of(prop.sharedMemPerBlockOptin); }

int ilog2_floor(int n) {
    int l = 0;
    while ((2 << l) <= n) ++l;
    return l;
}

// Shared memory of the kernels for one grid under a launch shape.
struct SmemNeed {
    size_t x, yz, slab, yfft, zdct;
};
SmemNeed smem_need(const ibf_grid &g, int mixed, const ibf_tuning &t) {
    const size_t csz = mixed ? 8 : 16, rsz = mixed ? 4 : 8;
    const int nx2 = g.nx / t.x_n1, ny2 = g.ny / t.y_n1;
    SmemNeed n{0, 0, 0, 0, 0};
    n.x = (size_t)(t.rows / 2) * (size_t)(t.x_n1 * (nx2 + 1) + 1) * csz;
    const size_t sstr = (size_t)(t.y_n1 * (ny2 + 1) + 1), nslot = (size_t)g.ny * t.mb;
    if (t.yz_kernel == 1) {  // layouts of k_yzfwd / k_yzbwd
        const size_t fwd = kYZStages * ((t.mb * sstr * csz + nslot * rsz + 15) & ~(size_t)15) + nslot * csz;
        const size_t bwd = kYZStages * ((nslot * (csz + rsz) + 15) & ~(size_t)15) + (t.mb * sstr + nslot) * csz;
        n.yz = std::max(fwd, bwd);
        if (mixed && t.mb == 1 && g.bc_y != IBF_BC_NEUMANN)
            n.yz = std::max(n.yz, std::max(yz_pipe_smem(g.ny, (int)sstr), yz_bulk_smem(g.ny, (int)sstr)));
    } else if (t.yz_kernel == 2) {
        n.slab = (((size_t)g.nz * t.mb * sstr * csz) + 15) & ~(size_t)15;
        if (t.tri > 1) n.slab += 3 * (size_t)g.nz * nslot * rsz;
    } else {
        n.yfft = (size_t)t.mb * sstr * csz;
        if (t.yz_kernel == 4) {  // k_zdct: zdct lines of the padded z sequence
            int a = 1, b = 1;
            factor(g.nz, &a, &b);
            n.zdct = (size_t)(mixed ? kZdctLinesF32 : kZdctLinesF64) * (size_t)(a * (b + 1) + 1) * csz;
        }
    }
    return n;
}

// z faces equally spaced (to 1e-12 of lz): the spectral-z path applies
bool z_uniform(const std::vector<double> &zf) {
    const int nz = (int)zf.size() - 1;
    const double lz = zf[nz] - zf[0];
    for (int k = 0; k <= nz; ++k)
        if (std::fabs(zf[k] - zf[0] - lz * (double)k / nz) > 1e-12 * lz) return false;
    return true;
}

bool fft_pair_ok(int n, int n1) { return n1 >= 1 && n % n1 == 0 && in_sizes(n1) && in_sizes(n / n1); }

// Fill the fields of `t` left <= 0 with the default launch shape of grid g and check
// the others.  The defaults: x kernels ~64 KB of FFT rows per CTA; balanced FFT
// factors; streaming y/z kernels with enough x-modes per block for 64+ FFT tasks per
// pass but at least one block per SM over the batch; Thomas with the pivot table.
ibf_status resolve_tuning(const ibf_grid &g, bool zuni, int mixed, long long total_cols, int nsm, size_t cap,
                          ibf_tuning *t) {
    const int nxh = x_modes(g);
    const int ny_even = (g.ny + 1) & ~1;
    int a = 1, b = 1;  // nx and ny factor (validate checked them)
    if (t->x_n1 <= 0) { factor(g.nx, &a, &b); t->x_n1 = a; }
    if (t->y_n1 <= 0) { factor(g.ny, &a, &b); t->y_n1 = a; }
    if (!fft_pair_ok(g.nx, t->x_n1) || !fft_pair_ok(g.ny, t->y_n1)) return IBF_ERR_UNSUPPORTED_SIZE;
    if (t->rows <= 0) {
        const int target = mixed ? 8192 : 4096;
        t->rows = std::max(2, std::min(2 * std::max(1, target / g.nx), ny_even));
    }
    if (t->rows & 1) return IBF_ERR_UNSUPPORTED_SIZE;
    t->rows = std::min(t->rows, std::max(2, ny_even));
    if (t->yz_kernel <= 0) t->yz_kernel = 1;
    if (t->yz_kernel > 4) return IBF_ERR_INVALID_ARG;
    if (t->yz_kernel == 4) {  // spectral z: uniform z, Neumann at both ends, nz = n1 n2 in the FFT sizes
        int a, b;
        if (!zuni || g.bc_zhi != IBF_BC_NEUMANN || !factor(g.nz, &a, &b)) return IBF_ERR_INVALID_ARG;
    }
    if (t->mb <= 0) {
        const int ny2 = g.ny / t->y_n1;
        const int mbmax = std::max(1, std::min(nxh, 4096 / g.ny));
        const int want = (64 + ny2 - 1) / ny2;
        // as few x-modes per block as keep every column block of the batch resident at
        // once (one wave), but no more than 64 FFT tasks per pass need
        const long long slots = (long long)(mixed ? kYZResidentF32 : kYZResidentF64) * nsm;
        t->mb = (int)std::min<long long>(std::min(mbmax, want), std::max<long long>(1, (total_cols + slots - 1) / slots));
    }
    t->mb = std::min(t->mb, nxh);
    if (t->tri <= 0) t->tri = 1;
    if (t->tri > 1 + ilog2_floor(g.nz)) return IBF_ERR_INVALID_ARG;
    const SmemNeed n = smem_need(g, mixed, *t);
    if (n.x > cap || n.yz > cap || n.slab > cap || n.yfft > cap || n.zdct > cap) return IBF_ERR_UNSUPPORTED_SIZE;
    return IBF_OK;
}

ibf_status build_plan(ibf_plan *pl, const ibf_grid *grids, int ngrids, const ibf_tuning *tuning) {
    const int mixed = pl->mixed;
    const size_t csz = mixed ? 8 : 16;   // complex element bytes
    const size_t rsz = mixed ? 4 : 8;    // real element bytes
    cudaDeviceProp prop;
    cudaError_t e = cudaGetDeviceProperties(&prop, pl->device);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetDeviceProperties");
    const int nsm = prop.multiProcessorCount;

    pl->grids.resize(ngrids);
    long long total_cols = 0;
    for (int g = 0; g < ngrids; ++g) total_cols += x_modes(grids[g]);

    long long spec = 0, cells = 0;
    int zoff = 0, poff = 0, xblk = 0, yzblk = 0, strblk = 0, slabblk = 0, yfftblk = 0, sweepblk = 0, zdctblk = 0;
    std::vector<int> str_start(ngrids + 1, 0), slab_start(ngrids + 1, 0), yfft_start(ngrids + 1, 0),
        sweep_start(ngrids + 1, 0), zdct_start(ngrids + 1, 0);
    std::vector<double> twx_all, twy_all, tmp;
    size_t maxx = 0, maxyz = 0, maxslab = 0, maxyfft = 0;
    for (int g = 0; g < ngrids; ++g) {
        GridHost &H = pl->grids[g];
        H.g = grids[g];
        IBF_TRY(validate_grid(&grids[g], H.zf));
        H.g.zf = nullptr;
        GridDev &d = H.d;
        memset(&d, 0, sizeof(d));
        d.nx = H.g.nx; d.ny = H.g.ny; d.nz = H.g.nz;
        d.nxh = x_modes(H.g);
        d.dir_top = H.g.bc_zhi == IBF_BC_DIRICHLET;
        d.wall_x = H.g.bc_x == IBF_BC_NEUMANN;
        d.wall_y = H.g.bc_y == IBF_BC_NEUMANN;
        d.nxu = d.nx + d.wall_x;
        d.nyv = d.ny + d.wall_y;
        ibf_tuning &t = H.tun;
        t = tuning ? tuning[g] : ibf_tuning{0, 0, 0, 0, 0, 0};
        IBF_TRY(resolve_tuning(H.g, z_uniform(H.zf), mixed, total_cols, nsm, smem_cap(prop), &t));
        d.nx1 = t.x_n1; d.nx2 = d.nx / t.x_n1;
        d.ny1 = t.y_n1; d.ny2 = d.ny / t.y_n1;
        d.mb = t.mb;
        d.ncb = (d.nxh + d.mb - 1) / d.mb;
        d.rows = t.rows;
        d.yzk = t.yz_kernel - 1;
        d.cr_levels = t.tri - 1;
        d.nrb = (d.ny + d.rows - 1) / d.rows;
        d.spec_off = spec;
        spec += (long long)d.nz * d.ncb * d.ny * d.mb;
        d.cell_off = cells;
        cells += (long long)d.nx * d.ny * d.nz;
        d.tab_off = d.spec_off;
        d.z_off = zoff;
        zoff += d.nz + 1;
        d.part_off = poff;
        poff += 2 * d.nz * d.nrb;  // room for the half-block split (xfwd_split)
        d.twx_off = (int)(twx_all.size() / 2);
        twiddles(d.nx, d.nx1, tmp);
        twx_all.insert(twx_all.end(), tmp.begin(), tmp.end());
        d.twy_off = (int)(twy_all.size() / 2);
        twiddles(d.ny, d.ny1, tmp);
        twy_all.insert(twy_all.end(), tmp.begin(), tmp.end());
        d.dctx_off = (int)(twx_all.size() / 2);
        if (d.wall_x) {
            dct_twiddles(d.nx, tmp);
            twx_all.insert(twx_all.end(), tmp.begin(), tmp.end());
        }
        d.dcty_off = (int)(twy_all.size() / 2);
        if (d.wall_y) {
            dct_twiddles(d.ny, tmp);
            twy_all.insert(twy_all.end(), tmp.begin(), tmp.end());
        }
        d.xblk_off = xblk;
        xblk += d.nz * d.nrb;
        d.yzblk_off = yzblk;
        yzblk += d.ncb;
        str_start[g] = strblk;
        slab_start[g] = slabblk;
        yfft_start[g] = yfftblk;
        sweep_start[g] = sweepblk;
        if (d.yzk == 0) {
            strblk += d.ncb;
        } else if (d.yzk == 1) {
            slabblk += d.ncb;
        } else {
            yfftblk += d.nz * d.ncb;
            if (d.yzk == 2)
                sweepblk += (int)(((long long)d.ncb * d.ny * d.mb + kSweepThreads - 1) / kSweepThreads);
        }
        zdct_start[g] = zdctblk;
        if (d.yzk == 3) {
            const int lines = mixed ? kZdctLinesF32 : kZdctLinesF64;
            zdctblk += (int)(((long long)d.ncb * d.ny * d.mb + lines - 1) / lines);
            factor(d.nz, &d.nz1, &d.nz2);
            d.fnz1 = make_fdiv(d.nz1);
            d.fnz2 = make_fdiv(d.nz2);
            d.twz_off = (int)(twy_all.size() / 2);
            twiddles(d.nz, d.nz1, tmp);
            twy_all.insert(twy_all.end(), tmp.begin(), tmp.end());
            d.dctz_off = (int)(twy_all.size() / 2);
            dct_twiddles(d.nz, tmp);
            twy_all.insert(twy_all.end(), tmp.begin(), tmp.end());
        }
        d.dx = H.g.lx / d.nx; d.dy = H.g.ly / d.ny;
        d.rdx = 1.0 / d.dx; d.rdy = 1.0 / d.dy;
        d.inv_nxy = 1.0 / ((double)d.nx * d.ny);
        d.sum_hz = H.zf[d.nz] - H.zf[0];
        d.fnx = make_fdiv(d.nx);
        d.fnph = make_fdiv(d.nx / 2 + 1);
        d.fnx1 = make_fdiv(d.nx1);
        d.fnx2 = make_fdiv(d.nx2);
        d.fny1 = make_fdiv(d.ny1);
        d.fny2 = make_fdiv(d.ny2);
        d.fmb = make_fdiv(d.mb);
        d.frows = make_fdiv(d.rows);
        d.fnpair = make_fdiv(d.rows / 2);
        d.fnpair2 = make_fdiv(std::max(1, d.rows / 4));
        {
            const SmemNeed n = smem_need(H.g, mixed, t);
            maxx = std::max(maxx, n.x);
            maxyz = std::max(maxyz, n.yz);
            maxslab = std::max(maxslab, n.slab);
            maxyfft = std::max(maxyfft, n.yfft);
            pl->zdctsmem = std::max(pl->zdctsmem, n.zdct);
            const size_t csz = mixed ? 8 : 16;
            pl->helmsmem = std::max(pl->helmsmem, (size_t)(yhelm_group(t.mb) * t.mb) *
                                                      (size_t)(t.y_n1 * (d.ny2 + 1) + 1) * csz);
        }
        pl->maxnz = std::max(pl->maxnz, d.nz);
        pl->total_cells += (long long)d.nx * d.ny * d.nz;
    }
    const size_t cap = smem_cap(prop);
    pl->smemcap = cap;
    if (maxx > cap || maxyz > cap || maxslab > cap || maxyfft > cap || pl->zdctsmem > cap ||
        (size_t)10 * (pl->maxnz + 1) * 8 > cap)
        return IBF_ERR_UNSUPPORTED_SIZE;
    str_start[ngrids] = strblk;
    slab_start[ngrids] = slabblk;
    yfft_start[ngrids] = yfftblk;
    sweep_start[ngrids] = sweepblk;
    zdct_start[ngrids] = zdctblk;
    pl->nzdctblk = zdctblk;
    pl->yfftsmem = maxyfft;
    pl->nyfftblk = yfftblk;
    pl->nsweepblk = sweepblk;
    pl->xsmem = maxx;
    pl->yzsmem = maxyz;
    pl->slabsmem = maxslab;
    pl->nxblk = xblk;
    pl->nyzblk = yzblk;
    pl->nstrblk = strblk;
    pl->nslabblk = slabblk;

    // per-level arrays
    const int nzt = zoff;
    std::vector<double> hz(nzt, 0.0), rhz(nzt, 0.0), rgzf(nzt, 0.0), az(nzt, 0.0), cz(nzt, 0.0), inv00(nzt, 0.0);
    std::vector<float> azf(nzt), czf(nzt);
    std::vector<float> rhz_df(2 * nzt), rgzf_df(2 * nzt);
    for (int g = 0; g < ngrids; ++g) {
        const GridHost &H = pl->grids[g];
        const int nz = H.d.nz, o = H.d.z_off;
        const std::vector<double> &zf = H.zf;
        for (int k = 0; k < nz; ++k) { hz[o + k] = zf[k + 1] - zf[k]; rhz[o + k] = 1.0 / hz[o + k]; }
        for (int k = 1; k < nz; ++k) {
            const double gz = 0.5 * (zf[k] + zf[k + 1]) - 0.5 * (zf[k - 1] + zf[k]);
            rgzf[o + k] = 1.0 / gz;
        }
        for (int k = 0; k < nz; ++k) {
            az[o + k] = rhz[o + k] * rgzf[o + k];
            cz[o + k] = rhz[o + k] * rgzf[o + k + 1];
        }
        if (H.d.dir_top) {
            // outlet face: phi = 0 there, so the flux through it couples level nz-1 to
            // the face value only (an extra diagonal term, no coupling coefficient)
            rgzf[o + nz] = 1.0 / (zf[nz] - 0.5 * (zf[nz - 1] + zf[nz]));
            pl->grids[g].d.ez_top = rhz[o + nz - 1] * rgzf[o + nz];
        }
        // pinned (0,0) system: level 0 fixed to zero
        double cp = 0.0;
        inv00[o] = 0.0;
        for (int k = 1; k < nz; ++k) {
            inv00[o + k] = 1.0 / (-(az[o + k] + cz[o + k]) - az[o + k] * cp);
            cp = cz[o + k] * inv00[o + k];
        }
        for (int k = 0; k <= nz; ++k) {
            azf[o + k] = (float)az[o + k];
            czf[o + k] = (float)cz[o + k];
            float h = (float)rhz[o + k];
            rhz_df[2 * (o + k)] = h;
            rhz_df[2 * (o + k) + 1] = (float)(rhz[o + k] - (double)h);
            h = (float)rgzf[o + k];
            rgzf_df[2 * (o + k)] = h;
            rgzf_df[2 * (o + k) + 1] = (float)(rgzf[o + k] - (double)h);
        }
    }

    // device allocations
    Work &w = pl->work;
    w.ngrids = ngrids;
    w.walls = 0;
    for (int g = 0; g < ngrids; ++g) w.walls |= pl->grids[g].d.wall_x | pl->grids[g].d.wall_y;
    w.xinv_split = mixed ? 1 : 0;
    for (int g = 0; g < ngrids; ++g)
        if (pl->grids[g].d.rows % 4 != 0) w.xinv_split = 0;
    w.xfwd_split = w.xinv_split;
    GridDev *dgrids;
    IBF_TRY(dalloc(pl, &dgrids, sizeof(GridDev) * ngrids));
    w.grids = dgrids;
    int *dx, *dyz, *dstr, *dslab, *dyfft, *dsweep, *dzdct;
    IBF_TRY(dalloc(pl, &dx, sizeof(int) * (ngrids + 1)));
    IBF_TRY(dalloc(pl, &dyz, sizeof(int) * (ngrids + 1)));
    IBF_TRY(dalloc(pl, &dstr, sizeof(int) * (ngrids + 1)));
    IBF_TRY(dalloc(pl, &dslab, sizeof(int) * (ngrids + 1)));
    IBF_TRY(dalloc(pl, &dyfft, sizeof(int) * (ngrids + 1)));
    IBF_TRY(dalloc(pl, &dsweep, sizeof(int) * (ngrids + 1)));
    IBF_TRY(dalloc(pl, &dzdct, sizeof(int) * (ngrids + 1)));
    w.yfft_start = dyfft;
    w.sweep_start = dsweep;
    w.zdct_start = dzdct;
    w.xblk_start = dx;
    w.yzblk_start = dyz;
    w.ystr_start = dstr;
    w.slab_start = dslab;
    IBF_TRY(dalloc(pl, &w.sol00, sizeof(double) * (size_t)zoff));
    IBF_TRY(dalloc(pl, &w.z.hz, sizeof(double) * nzt));
    IBF_TRY(dalloc(pl, &w.z.rhz, sizeof(double) * nzt));
    IBF_TRY(dalloc(pl, &w.z.rgzf, sizeof(double) * nzt));
    IBF_TRY(dalloc(pl, &w.z.az, sizeof(double) * nzt));
    IBF_TRY(dalloc(pl, &w.z.cz, sizeof(double) * nzt));
    IBF_TRY(dalloc(pl, &w.z.inv00, sizeof(double) * nzt));
    IBF_TRY(dalloc(pl, &w.z.azf, sizeof(float) * nzt));
    IBF_TRY(dalloc(pl, &w.z.czf, sizeof(float) * nzt));
    IBF_TRY(dalloc(pl, &w.z.rhz_df, sizeof(float2) * nzt));
    IBF_TRY(dalloc(pl, &w.z.rgzf_df, sizeof(float2) * nzt));
    IBF_TRY(dalloc(pl, &pl->helm, sizeof(double) * 6 * (size_t)nzt));
    IBF_TRY(dalloc(pl, &pl->helmf, sizeof(float) * 6 * (size_t)nzt));
    {
        long long nf = 0;
        pl->fxy_off.resize(ngrids);
        for (int g = 0; g < ngrids; ++g) {
            pl->fxy_off[g] = nf;
            nf += pl->grids[g].d.nxh + pl->grids[g].d.ny;
        }
        IBF_TRY(dalloc(pl, &pl->fxy, sizeof(double) * (size_t)nf));
        IBF_TRY(dalloc(pl, &pl->fxyf, sizeof(float) * (size_t)nf));
        IBF_TRY(dalloc(pl, &pl->fxy_off_dev, sizeof(long long) * (size_t)ngrids));
        IBF_TRY(upload(pl->fxy_off.data(), pl->fxy_off_dev, sizeof(long long) * (size_t)ngrids));
    }
    IBF_TRY(dalloc(pl, &w.spec, csz * (size_t)spec));
    IBF_TRY(dalloc(pl, &w.tab, rsz * (size_t)spec));
    void *twx, *twy;
    IBF_TRY(dalloc(pl, &twx, csz * twx_all.size() / 2));
    IBF_TRY(dalloc(pl, &twy, csz * twy_all.size() / 2));
    w.twx = twx;
    w.twy = twy;
    if (!mixed && pl->opts.pressure == IBF_P_IMPLICIT) IBF_TRY(dalloc(pl, &w.bws, sizeof(double) * (size_t)cells));
    if (mixed) {
        IBF_TRY(dalloc(pl, &w.bdf, sizeof(float2) * (size_t)cells));
        IBF_TRY(dalloc(pl, &w.phi_hi, sizeof(float) * (size_t)cells));
        IBF_TRY(dalloc(pl, &w.phi_lo, sizeof(float) * (size_t)cells));
        if (pl->opts.refine_steps >= 2) {
            IBF_TRY(dalloc(pl, &w.phi_lo2, sizeof(float) * (size_t)cells));
            // test hook: IBF_NO_KEPT_RESIDUAL makes the second sweep form its residual from
            // phi (b - <b> - L(phi_0 + delta_1)) instead of from the kept first residual
            const char *nokeep = getenv("IBF_NO_KEPT_RESIDUAL");
            if (!(nokeep && atoi(nokeep) > 0)) IBF_TRY(dalloc(pl, &w.rdf, sizeof(float2) * (size_t)cells));
        }
        // test hook: IBF_FAULT_LOSE_COPY makes the round-based forward y/z kernel drop one
        // plane copy, so that its bounded wait runs out and IBF_ERR_TIMEOUT is reported
        const char *lose = getenv("IBF_FAULT_LOSE_COPY");
        w.fault_lose_copy = (lose && atoi(lose) > 0) ? 1 : 0;
    } else {
        IBF_TRY(dalloc(pl, &w.phi_ws, sizeof(double) * (size_t)cells));
    }
    IBF_TRY(dalloc(pl, &w.partial, sizeof(double) * (size_t)std::max(poff, 1)));
    IBF_TRY(dalloc(pl, &w.partial_phi, sizeof(double) * (size_t)std::max(poff, 1)));
    IBF_TRY(dalloc(pl, &w.mean_b, sizeof(double) * ngrids));
    IBF_TRY(dalloc(pl, &w.maxb, sizeof(unsigned long long) * ngrids));
    IBF_TRY(dalloc(pl, &w.maxdiv, sizeof(unsigned long long) * ngrids));
    IBF_TRY(dalloc(pl, &w.err, sizeof(unsigned)));

    std::vector<GridDev> hd(ngrids);
    std::vector<int> xs(ngrids + 1), ys(ngrids + 1);
    for (int g = 0; g < ngrids; ++g) {
        hd[g] = pl->grids[g].d;
        xs[g] = hd[g].xblk_off;
        ys[g] = hd[g].yzblk_off;
    }
    xs[ngrids] = xblk;
    ys[ngrids] = yzblk;
    IBF_TRY(upload(hd.data(), dgrids, sizeof(GridDev) * ngrids));
    IBF_TRY(upload(xs.data(), dx, sizeof(int) * (ngrids + 1)));
    IBF_TRY(upload(ys.data(), dyz, sizeof(int) * (ngrids + 1)));
    IBF_TRY(upload(str_start.data(), dstr, sizeof(int) * (ngrids + 1)));
    IBF_TRY(upload(slab_start.data(), dslab, sizeof(int) * (ngrids + 1)));
    IBF_TRY(upload(yfft_start.data(), dyfft, sizeof(int) * (ngrids + 1)));
    IBF_TRY(upload(sweep_start.data(), dsweep, sizeof(int) * (ngrids + 1)));
    IBF_TRY(upload(zdct_start.data(), dzdct, sizeof(int) * (ngrids + 1)));
    IBF_TRY(upload(hz.data(), w.z.hz, sizeof(double) * nzt));
    IBF_TRY(upload(rhz.data(), w.z.rhz, sizeof(double) * nzt));
    IBF_TRY(upload(rgzf.data(), w.z.rgzf, sizeof(double) * nzt));
    IBF_TRY(upload(az.data(), w.z.az, sizeof(double) * nzt));
    IBF_TRY(upload(cz.data(), w.z.cz, sizeof(double) * nzt));
    IBF_TRY(upload(inv00.data(), w.z.inv00, sizeof(double) * nzt));
    IBF_TRY(upload(azf.data(), w.z.azf, sizeof(float) * nzt));
    IBF_TRY(upload(czf.data(), w.z.czf, sizeof(float) * nzt));
    IBF_TRY(upload(rhz_df.data(), w.z.rhz_df, sizeof(float2) * nzt));
    IBF_TRY(upload(rgzf_df.data(), w.z.rgzf_df, sizeof(float2) * nzt));
    if (mixed) {
        std::vector<float> fx(twx_all.begin(), twx_all.end()), fy(twy_all.begin(), twy_all.end());
        IBF_TRY(upload(fx.data(), twx, sizeof(float) * fx.size()));
        IBF_TRY(upload(fy.data(), twy, sizeof(float) * fy.size()));
    } else {
        IBF_TRY(upload(twx_all.data(), twx, sizeof(double) * twx_all.size()));
        IBF_TRY(upload(twy_all.data(), twy, sizeof(double) * twy_all.size()));
    }
    e = cudaMemset(w.spec, 0, csz * (size_t)spec);
    if (e != cudaSuccess) return cuda_fail(e, "cudaMemset");
    e = cudaMemset(w.err, 0, sizeof(unsigned));
    if (e != cudaSuccess) return cuda_fail(e, "cudaMemset");
    e = cudaMemset(w.mean_b, 0, sizeof(double) * ngrids);
    if (e != cudaSuccess) return cuda_fail(e, "cudaMemset");

    e = set_smem_limits(mixed);
    if (e == cudaSuccess) e = set_smem_limits_visc(mixed);
    if (e != cudaSuccess) return cuda_fail(e, "cudaFuncSetAttribute");
    e = launch_build_table(mixed, w, pl->nyzblk, nullptr);
    if (e != cudaSuccess) return cuda_fail(e, "pivot table kernel");
    e = cudaDeviceSynchronize();
    if (e != cudaSuccess) return cuda_fail(e, "pivot table kernel");
    return IBF_OK;
}

// ------------------------------------------------------------ call sequencing
struct Ctx {
    ibf_plan *pl;
    cudaStream_t st;
};

cudaEvent_t get_event(ibf_plan *pl) {
    if (!pl->ev_pool.empty()) {
        cudaEvent_t e = pl->ev_pool.back();
        pl->ev_pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    cudaEventCreate(&e);
    return e;
}

template <typename F> ibf_status timed(Ctx &c, const char *name, F f) {
    ProfRec r{name, nullptr, nullptr};
    if (c.pl->prof) {
        r.e0 = get_event(c.pl);
        r.e1 = get_event(c.pl);
        cudaEventRecord(r.e0, c.st);
    }
    cudaError_t e = f();
    if (c.pl->prof) {
        cudaEventRecord(r.e1, c.st);
        c.pl->prof_pending.push_back(r);
    }
    if (e != cudaSuccess) return cuda_fail(e, name);
    return IBF_OK;
}

// Fill user pointers for grids [g0, g1).
void fill_ptrs(ibf_plan *pl, UserPtrs &p, int g0, int g1, const ibf_fields *in, const ibf_fields *out) {
    memset(&p, 0, sizeof(p));
    p.g0 = g0;
    p.g1 = g1;
    p.blk0 = pl->grids[g0].d.xblk_off;
    for (int g = g0; g < g1; ++g) {
        const int i = g - g0;
        if (in) {
            p.in_u[i] = in[g].u; p.in_v[i] = in[g].v; p.in_w[i] = in[g].w; p.in_p[i] = in[g].p;
            p.in_q[i] = in[g].q;
        }
        if (out) { p.out_u[i] = out[g].u; p.out_v[i] = out[g].v; p.out_w[i] = out[g].w; p.out_p[i] = out[g].p; }
    }
}

int chunk_blocks(ibf_plan *pl, int g0, int g1) {
    const int b0 = pl->grids[g0].d.xblk_off;
    const int b1 = (g1 < pl->ngrids) ? pl->grids[g1].d.xblk_off : pl->nxblk;
    return b1 - b0;
}

// x-kernel launches over chunks of grids (user pointers travel as launch parameters)
template <typename F>
ibf_status for_chunks(Ctx &c, const char *name, const ibf_fields *in, const ibf_fields *out, F f) {
    for (int g0 = 0; g0 < c.pl->ngrids; g0 += kGridsPerLaunch) {
        const int g1 = std::min(c.pl->ngrids, g0 + kGridsPerLaunch);
        UserPtrs p;
        fill_ptrs(c.pl, p, g0, g1, in, out);
        const int nb = chunk_blocks(c.pl, g0, g1);
        IBF_TRY(timed(c, name, [&]() { return f(p, nb); }));
    }
    return IBF_OK;
}

// One solve S^-1 of the right-hand side already transformed into the spectrum.
ibf_status solve_core(Ctx &c, int first) {
    ibf_plan *pl = c.pl;
    const Work &w = pl->work;
    if (pl->nstrblk > 0)
        IBF_TRY(timed(c, "yz_forward", [&]() { return launch_yzfwd(pl->mixed, w, pl->nstrblk, pl->yzsmem, c.st); }));
    if (pl->nyfftblk > 0) {
        IBF_TRY(timed(c, "y_fft_forward", [&]() { return launch_yfft(pl->mixed, 0, w, pl->nyfftblk, pl->yfftsmem, c.st); }));
        if (pl->nsweepblk > 0)
            IBF_TRY(timed(c, "z_sweep_forward", [&]() { return launch_zsweep(pl->mixed, 0, w, pl->nsweepblk, c.st); }));
    }
    if (pl->nzdctblk > 0)  // spectral z: DCT along z, division, inverse DCT (before k_00 writes the (0,0) column)
        IBF_TRY(timed(c, "z_dct_solve", [&]() { return launch_zdct(pl->mixed, w, pl->nzdctblk, pl->zdctsmem, c.st); }));
    IBF_TRY(timed(c, "mode00", [&]() { return launch_k00(w, pl->mixed, first, pl->maxnz, c.st); }));
    if (pl->nstrblk > 0)
        IBF_TRY(timed(c, "yz_backward", [&]() { return launch_yzbwd(pl->mixed, w, pl->nstrblk, pl->yzsmem, c.st); }));
    if (pl->nyfftblk > 0) {
        if (pl->nsweepblk > 0)
            IBF_TRY(timed(c, "z_sweep_backward", [&]() { return launch_zsweep(pl->mixed, 1, w, pl->nsweepblk, c.st); }));
        IBF_TRY(timed(c, "y_fft_inverse", [&]() { return launch_yfft(pl->mixed, 1, w, pl->nyfftblk, pl->yfftsmem, c.st); }));
    }
    if (pl->nslabblk > 0)
        IBF_TRY(timed(c, "yz_slab", [&]() { return launch_yzslab(pl->mixed, w, pl->nslabblk, pl->slabsmem, c.st); }));
    return IBF_OK;
}

ibf_status run(ibf_plan *pl, const ibf_fields *in, const ibf_fields *out, double dt, double alpha,
               const ibf_stats *stats, cudaStream_t st, int adjoint) {
    Ctx c{pl, st};
    const Work &w = pl->work;
    const double s = alpha * dt, rs = 1.0 / s;
    const int mixed = pl->mixed;
    // fp64 path: the adjoint's phi, and phi under a pressure update, live in the plan;
    // mixed path: phi is refined as float-float in the plan and written out by the
    // correction kernel.
    const int pmode = adjoint ? 0 : pl->opts.pressure;
    const int use_ws = (adjoint || pmode) ? 1 : 0;
    const double cimp = pmode == IBF_P_IMPLICIT ? 0.5 * alpha * dt * pl->opts.inv_re : 0.0;
    const int R = mixed ? pl->opts.refine_steps : 0;
    cudaError_t e = cudaMemsetAsync(w.maxb, 0, sizeof(unsigned long long) * pl->ngrids, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(w.maxdiv, 0, sizeof(unsigned long long) * pl->ngrids, st);
    if (e != cudaSuccess) return cuda_fail(e, "cudaMemsetAsync");
    bool has_q = false;  // mass sources enter the forward map only (the adjoint is of u* -> (u, phi))
    for (int g = 0; g < pl->ngrids && !adjoint; ++g) has_q |= in[g].q != nullptr;
    const int xmode = adjoint ? XM_ADJ : (has_q ? XM_DIVQ : XM_DIV);
    IBF_TRY(for_chunks(c, adjoint ? "x_forward_adjoint_rhs" : "x_forward_div", in, out, [&](const UserPtrs &p, int nb) {
        return launch_xfwd(mixed, xmode, w, p, use_ws, 0, nb, s, rs, pl->xsmem, st);
    }));
    IBF_TRY(solve_core(c, 1));
    IBF_TRY(for_chunks(c, "x_inverse_store", in, out, [&](const UserPtrs &p, int nb) {
        return launch_xinv(mixed, IM_STORE, w, p, use_ws, 0, nb, pl->xsmem, st);
    }));
    // Sweep r adds its correction delta to phi: the first into the low word of the pair
    // (phi_0, delta), the middle ones by an exact renormalising sum, the last one (two or
    // more sweeps) into phi_lo2, which the correction kernel adds to the pair.
    const int lo2 = R >= 2;
    for (int r = 0; r < R; ++r) {
        const int lo_valid = r > 0;
        const bool last = lo2 && r == R - 1;
        // the first sweep's kernels (phi_0 plain fp32) and the later ones' (float-float
        // phi) are profiled under their own names
        IBF_TRY(for_chunks(c, lo_valid ? "x_forward_residual2" : "x_forward_residual", in, out,
                           [&](const UserPtrs &p, int nb) {
            // the second sweep starts from the first sweep's stored residual
            return launch_xfwd(mixed, (r == 1 && w.rdf) ? XM_RESID1 : XM_RESID, w, p, use_ws, lo_valid, nb, s, rs,
                               pl->xsmem, st);
        }));
        IBF_TRY(solve_core(c, 0));
        IBF_TRY(for_chunks(c, last ? "x_inverse_last" : (lo_valid ? "x_inverse_accumulate2" : "x_inverse_accumulate"),
                           in, out, [&](const UserPtrs &p, int nb) {
            return launch_xinv(mixed, last ? IM_LAST : IM_ACCUM, w, p, use_ws, lo_valid, nb, pl->xsmem, st);
        }));
    }
    IBF_TRY(for_chunks(c, adjoint ? "correct_adjoint" : "correct", in, out, [&](const UserPtrs &p, int nb) {
        return launch_correct(mixed, adjoint, w, p, use_ws, R > 0, lo2, nb, s, pmode, cimp, st);
    }));
    if (!adjoint && stats && (stats->max_div || stats->max_div_in || stats->compat)) {
        if (stats->max_div) {
            IBF_TRY(for_chunks(c, "divergence_stat", in, out, [&](const UserPtrs &p, int nb) {
                return launch_divstat(mixed, w, p, nb, st);
            }));
        }
        IBF_TRY(timed(c, "finalize", [&]() {
            return launch_finalize(w, stats->max_div, stats->max_div_in, stats->compat, s, st);
        }));
    }
    pl->last_stream = st;
    return IBF_OK;
}

bool fields_ok(const ibf_fields *f, int n, bool need_p) {
    if (!f) return false;
    for (int g = 0; g < n; ++g) {
        if (!f[g].u || !f[g].v || !f[g].w) return false;
        if (need_p && !f[g].p) return false;
    }
    return true;
}

// Plan construction with resolved launch shapes (tuning: ngrids entries).
ibf_status make_plan(ibf_plan **plan, const ibf_grid *grids, int ngrids, const ibf_opts *opts, int device,
                     const ibf_tuning *tuning) {
    ibf_plan *pl = new (std::nothrow) ibf_plan();
    if (!pl) return IBF_ERR_OOM;
    pl->device = device;
    pl->ngrids = ngrids;
    pl->opts = *opts;
    pl->mixed = opts->precision == IBF_MIXED;
    ibf_status s = build_plan(pl, grids, ngrids, tuning);
    if (s != IBF_OK) {
        cudaDeviceSynchronize();
        free_all(pl);
        delete pl;
        return s;
    }
    *plan = pl;
    return IBF_OK;
}

// ------------------------------------------------------------ autotuner
// Candidate launch shapes of one grid are timed as whole projections (one-grid plan,
// zero fields, one warm-up and three timed calls on a private stream), by coordinate
// descent: x-FFT factors, x rows per CTA, y-FFT factors, then the y/z kernel (streaming
// with each column-block width; resident slab with each width and tridiagonal
// algorithm that fits shared memory).  Results are cached per (shape, boundary
// conditions, precision, refinement, forced fields) for the life of the process.
struct TuneKey {
    int v[15];
    bool operator<(const TuneKey &o) const { return std::lexicographical_compare(v, v + 15, o.v, o.v + 15); }
};
std::mutex g_tune_mu;
std::map<TuneKey, ibf_tuning> g_tune_cache;

struct TuneBench {
    int device;
    ibf_opts opts;
    ibf_grid g;
    ibf_fields in, out;
    cudaStream_t st = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
};

// projection time of grid b.g under shape t (ms), or a negative value if the shape
// is not feasible
float time_shape(TuneBench &b, const ibf_tuning &t) {
    ibf_plan *p = nullptr;
    if (make_plan(&p, &b.g, 1, &b.opts, b.device, &t) != IBF_OK) {
        g_last_error.clear();
        return -1.f;
    }
    float best = -1.f;
    if (run(p, &b.in, &b.out, 1e-3, 1.0, nullptr, b.st, 0) == IBF_OK && cudaStreamSynchronize(b.st) == cudaSuccess) {
        cudaEventRecord(b.e0, b.st);
        bool ok = true;
        for (int r = 0; r < 3 && ok; ++r) ok = run(p, &b.in, &b.out, 1e-3, 1.0, nullptr, b.st, 0) == IBF_OK;
        cudaEventRecord(b.e1, b.st);
        float ms = 0.f;
        if (ok && cudaEventSynchronize(b.e1) == cudaSuccess && cudaEventElapsedTime(&ms, b.e0, b.e1) == cudaSuccess)
            best = ms / 3.f;
    }
    cudaStreamSynchronize(b.st);
    (void)cudaGetLastError();
    free_all(p);
    delete p;
    return best;
}

ibf_status tune_grid(const ibf_grid &g, const ibf_opts &opts, int device, ibf_tuning *t) {
    std::vector<double> zf;
    IBF_TRY(validate_grid(&g, zf));
    const bool zuni = z_uniform(zf);
    TuneKey key;
    const int kv[15] = {g.nx, g.ny, g.nz, g.bc_x, g.bc_y, g.bc_zhi, opts.precision, opts.refine_steps,
                        t->rows, t->x_n1, t->y_n1, t->yz_kernel, t->mb, t->tri, zuni ? 1 : 0};
    std::copy(kv, kv + 15, key.v);
    {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        auto it = g_tune_cache.find(key);
        if (it != g_tune_cache.end()) { *t = it->second; return IBF_OK; }
    }
    const ibf_tuning forced = *t;
    TuneBench b;
    b.device = device;
    b.opts = opts;
    b.opts.autotune = 0;
    b.g = g;
    const size_t nxu = g.nx + (g.bc_x == IBF_BC_NEUMANN), nyv = g.ny + (g.bc_y == IBF_BC_NEUMANN);
    const size_t bu = 8 * (size_t)g.nz * g.ny * nxu, bv = 8 * (size_t)g.nz * nyv * g.nx,
                 bw = 8 * (size_t)(g.nz + 1) * g.ny * g.nx, bp = 8 * (size_t)g.nz * g.ny * g.nx;
    double *buf = nullptr;
    cudaError_t e = cudaMalloc(&buf, 2 * (bu + bv + bw) + bp);
    if (e != cudaSuccess) { (void)cudaGetLastError(); g_last_error = "autotune: cudaMalloc"; return IBF_ERR_OOM; }
    unsigned char *c = reinterpret_cast<unsigned char *>(buf);
    b.in = {(double *)c, (double *)(c + bu), (double *)(c + bu + bv), nullptr};
    c += bu + bv + bw;
    b.out = {(double *)c, (double *)(c + bu), (double *)(c + bu + bv), (double *)(c + bu + bv + bw)};
    e = cudaMemset(buf, 0, 2 * (bu + bv + bw) + bp);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&b.st, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreate(&b.e0);
    if (e == cudaSuccess) e = cudaEventCreate(&b.e1);
    ibf_status status = IBF_OK;
    if (e != cudaSuccess) status = cuda_fail(e, "autotune setup");

    ibf_tuning best = forced;
    float tbest = -1.f;
    static const bool log = getenv("IBF_AUTOTUNE_LOG") != nullptr;  // print every timed candidate
    auto consider = [&](ibf_tuning cand) {
        const float ms = time_shape(b, cand);
        if (log)
            fprintf(stderr, "ibf autotune %dx%dx%d: rows %d x_n1 %d y_n1 %d yz_kernel %d mb %d tri %d -> %.4f ms\n",
                    g.nx, g.ny, g.nz, cand.rows, cand.x_n1, cand.y_n1, cand.yz_kernel, cand.mb, cand.tri, ms);
        if (ms > 0.f && (tbest < 0.f || ms < tbest)) { tbest = ms; best = cand; }
    };
    if (status == IBF_OK) {
        {   // starting point: the defaults of the fields left free
            cudaDeviceProp prop;
            cudaGetDeviceProperties(&prop, device);
            ibf_tuning d = forced;
            if (resolve_tuning(g, zuni, opts.precision == IBF_MIXED, x_modes(g), prop.multiProcessorCount,
                               smem_cap(prop), &d) == IBF_OK)
                consider(d);
        }
        if (tbest > 0.f) {
            static const int kRows[] = {2, 4, 8, 16, 32, 64};
            static const int kMb[] = {1, 2, 4, 8, 16, 32};
            if (forced.x_n1 <= 0)
                for (int n1 : kFftSizes)
                    if (n1 != best.x_n1 && fft_pair_ok(g.nx, n1)) { ibf_tuning c2 = best; c2.x_n1 = n1; consider(c2); }
            if (forced.rows <= 0)
                for (int r : kRows)
                    if (r != best.rows && r <= ((g.ny + 1) & ~1)) { ibf_tuning c2 = best; c2.rows = r; consider(c2); }
            if (forced.y_n1 <= 0)
                for (int n1 : kFftSizes)
                    if (n1 != best.y_n1 && fft_pair_ok(g.ny, n1)) { ibf_tuning c2 = best; c2.y_n1 = n1; consider(c2); }
            const ibf_tuning base = best;
            const int nxh = x_modes(g);
            int a1, b1;
            const bool spectral_ok = zuni && g.bc_zhi == IBF_BC_NEUMANN && factor(g.nz, &a1, &b1);
            for (int kern = 1; kern <= 4; ++kern) {
                if (forced.yz_kernel > 0 && forced.yz_kernel != kern) continue;
                if (kern == 4 && !spectral_ok) continue;
                for (int mb : kMb) {
                    if (mb > nxh && mb != 1) continue;
                    if (forced.mb > 0 && forced.mb != mb) continue;
                    // slab: Thomas, 1-2 reduction levels, full reduction
                    const int ntri = kern == 2 ? 1 + ilog2_floor(g.nz) : 1;
                    for (int tri = 1; tri <= ntri; ++tri) {
                        if (forced.tri > 0 && forced.tri != tri) continue;
                        if (kern == 2 && tri > 3 && tri != ntri) continue;
                        ibf_tuning c2 = base;
                        c2.yz_kernel = kern;
                        c2.mb = mb;
                        c2.tri = tri;
                        if (c2.yz_kernel == base.yz_kernel && c2.mb == base.mb && c2.tri == base.tri) continue;
                        consider(c2);
                    }
                }
            }
        } else {
            status = IBF_ERR_UNSUPPORTED_SIZE;
        }
    }
    if (b.e0) cudaEventDestroy(b.e0);
    if (b.e1) cudaEventDestroy(b.e1);
    if (b.st) cudaStreamDestroy(b.st);
    cudaFree(buf);
    if (status != IBF_OK) return status;
    *t = best;
    std::lock_guard<std::mutex> lk(g_tune_mu);
    g_tune_cache[key] = best;
    return IBF_OK;
}

ibf_status autotune(const ibf_grid *grids, int ngrids, const ibf_opts &opts, int device, ibf_tuning *tun) {
    for (int g = 0; g < ngrids; ++g) IBF_TRY(tune_grid(grids[g], opts, device, &tun[g]));
    return IBF_OK;
}

}  // namespace

extern "C" {

const char *ibf_status_string(ibf_status s) {
    switch (s) {
        case IBF_OK: return "ok";
        case IBF_ERR_INVALID_ARG: return "invalid argument";
        case IBF_ERR_UNSUPPORTED_SIZE: return "unsupported grid size";
        case IBF_ERR_OOM: return "device allocation failed";
        case IBF_ERR_CUDA: return "CUDA runtime error";
        case IBF_ERR_TIMEOUT: return "bounded device wait timed out";
        case IBF_ERR_NONFINITE: return "non-finite value in the right-hand side";
        case IBF_WARN_INCOMPATIBLE_RHS: return "right-hand side incompatible with the Neumann walls (mean removed)";
        case IBF_ERR_UNSUPPORTED_BC: return "unsupported boundary condition";
    }
    return "unknown status";
}

const char *ibf_last_error(void) { return g_last_error.c_str(); }

ibf_status ibf_projection_plan(ibf_plan **plan, const ibf_grid *grids, int ngrids, const ibf_opts *opts, int device) {
    return ibf_projection_plan_tuned(plan, grids, ngrids, opts, device, nullptr);
}

ibf_status ibf_projection_plan_tuned(ibf_plan **plan, const ibf_grid *grids, int ngrids, const ibf_opts *opts,
                                     int device, const ibf_tuning *tuning) {
    if (!plan) return IBF_ERR_INVALID_ARG;
    *plan = nullptr;
    if (!grids || !opts || ngrids < 1 || ngrids > IBF_MAX_GRIDS || device < 0) return IBF_ERR_INVALID_ARG;
    if (opts->precision != IBF_FP64 && opts->precision != IBF_MIXED) return IBF_ERR_INVALID_ARG;
    if (opts->refine_steps < 0 || opts->refine_steps > 8) return IBF_ERR_INVALID_ARG;
    if (opts->pressure < IBF_P_PHI || opts->pressure > IBF_P_IMPLICIT || !std::isfinite(opts->inv_re) ||
        opts->inv_re < 0)
        return IBF_ERR_INVALID_ARG;
    if (opts->precision == IBF_FP64 && opts->refine_steps != 0) return IBF_ERR_INVALID_ARG;
    // host-side validation of every grid before touching the device
    for (int g = 0; g < ngrids; ++g) {
        std::vector<double> zf;
        ibf_status s = validate_grid(&grids[g], zf);
        if (s != IBF_OK) return s;
        if (tuning) {
            const ibf_tuning &t = tuning[g];
            if (t.yz_kernel > 4 || (t.rows > 0 && (t.rows & 1))) return IBF_ERR_INVALID_ARG;
            int a, b;
            if (t.yz_kernel == 4 &&
                (!z_uniform(zf) || grids[g].bc_zhi != IBF_BC_NEUMANN || !factor(grids[g].nz, &a, &b)))
                return IBF_ERR_INVALID_ARG;  // spectral z: uniform z, Neumann top, nz a product of FFT sizes
        }
    }
    cudaError_t e = cudaSetDevice(device);
    if (e != cudaSuccess) return cuda_fail(e, "cudaSetDevice");
    std::vector<ibf_tuning> tun(ngrids, ibf_tuning{0, 0, 0, 0, 0, 0});
    if (tuning) std::copy(tuning, tuning + ngrids, tun.begin());
    if (opts->autotune) IBF_TRY(autotune(grids, ngrids, *opts, device, tun.data()));
    return make_plan(plan, grids, ngrids, opts, device, tun.data());
}

ibf_status ibf_plan_get_tuning(const ibf_plan *plan, int g, ibf_tuning *out) {
    if (!plan || !out || g < 0 || g >= plan->ngrids) return IBF_ERR_INVALID_ARG;
    *out = plan->grids[g].tun;
    return IBF_OK;
}

ibf_status ibf_project(ibf_plan *plan, const ibf_fields *in, const ibf_fields *out, double dt, double alpha,
                       const ibf_stats *stats, void *stream) {
    if (!plan || !fields_ok(in, plan->ngrids, plan->opts.pressure != IBF_P_PHI) || !fields_ok(out, plan->ngrids, true))
        return IBF_ERR_INVALID_ARG;
    if (!(dt > 0) || !(alpha > 0) || !std::isfinite(dt) || !std::isfinite(alpha)) return IBF_ERR_INVALID_ARG;
    cudaError_t e = cudaSetDevice(plan->device);
    if (e != cudaSuccess) return cuda_fail(e, "cudaSetDevice");
    return run(plan, in, out, dt, alpha, stats, static_cast<cudaStream_t>(stream), 0);
}

ibf_status ibf_project_backward(ibf_plan *plan, const ibf_fields *grad_out, const ibf_fields *grad_in, double dt,
                                double alpha, void *stream) {
    if (!plan || !fields_ok(grad_out, plan->ngrids, false) || !fields_ok(grad_in, plan->ngrids, false))
        return IBF_ERR_INVALID_ARG;
    if (!(dt > 0) || !(alpha > 0) || !std::isfinite(dt) || !std::isfinite(alpha)) return IBF_ERR_INVALID_ARG;
    cudaError_t e = cudaSetDevice(plan->device);
    if (e != cudaSuccess) return cuda_fail(e, "cudaSetDevice");
    return run(plan, grad_out, grad_in, dt, alpha, nullptr, static_cast<cudaStream_t>(stream), 1);
}

ibf_status ibf_viscous_solve(ibf_plan *plan, const ibf_fields *in, const ibf_fields *out, double beta,
                             void *stream) {
    if (!plan || !fields_ok(in, plan->ngrids, false) || !fields_ok(out, plan->ngrids, false)) return IBF_ERR_INVALID_ARG;
    if (!(beta >= 0) || !std::isfinite(beta)) return IBF_ERR_INVALID_ARG;
    for (int g = 0; g < plan->ngrids; ++g)
        if (plan->grids[g].d.wall_x || plan->grids[g].d.wall_y) {
            g_last_error = "viscous solve: x and y must be periodic";
            return IBF_ERR_UNSUPPORTED_BC;
        }
    if (plan->helmsmem > plan->smemcap) {
        g_last_error = "viscous solve: the y transform of a column block does not fit in shared memory";
        return IBF_ERR_UNSUPPORTED_SIZE;
    }
    cudaError_t e = cudaSetDevice(plan->device);
    if (e != cudaSuccess) return cuda_fail(e, "cudaSetDevice");
    ibf_plan *pl = plan;
    Ctx c{pl, static_cast<cudaStream_t>(stream)};
    const Work &w = pl->work;
    const int mixed = pl->mixed;
    // the pivots and factors depend on beta only: rebuilt when it changes, and always
    // inside a stream capture (the graph then carries its own tables)
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(c.st, &cap) != cudaSuccess) return cuda_fail(cudaGetLastError(), "cudaStreamIsCapturing");
    if (!pl->helm_valid || pl->helm_beta != beta || cap != cudaStreamCaptureStatusNone) {
        IBF_TRY(timed(c, "helm_table", [&]() {
            return launch_helm_table(w, pl->ngrids, beta, pl->helm, pl->helmf, pl->fxy_off_dev, pl->fxy, pl->fxyf,
                                     c.st);
        }));
        pl->helm_valid = true;
        pl->helm_beta = beta;
    }
    // one velocity component at a time: x-FFT of the field, the x and y factors between
    // the y transforms, inverse x-FFT into the per-cell workspace, Thomas along z
    for (int comp = 0; comp < 3; ++comp) {
        std::vector<ibf_fields> cin(pl->ngrids);
        for (int g = 0; g < pl->ngrids; ++g) {
            cin[g] = ibf_fields{};
            cin[g].u = const_cast<double *>(comp == 0 ? in[g].u : (comp == 1 ? in[g].v : in[g].w));
            cin[g].v = cin[g].w = cin[g].u;
        }
        for (int g0 = 0; g0 < pl->ngrids; g0 += kGridsPerLaunch) {
            const int g1 = std::min(pl->ngrids, g0 + kGridsPerLaunch);
            UserPtrs p;
            fill_ptrs(pl, p, g0, g1, cin.data(), nullptr);
            p.zshift = comp == 2;
            const int nb = chunk_blocks(pl, g0, g1);
            IBF_TRY(timed(c, "viscous_x_forward", [&]() {
                return launch_xfwd(mixed, XM_COPY, w, p, 1, 0, nb, 1.0, 1.0, pl->xsmem, c.st);
            }));
        }
        for (int g = 0; g < pl->ngrids; ++g) {
            const GridDev &d = pl->grids[g].d;
            IBF_TRY(timed(c, "viscous_y", [&]() {
                const int gb = yhelm_group(d.mb);
                return launch_yhelm(mixed, w, g, d.nz * ((d.ncb + gb - 1) / gb), gb, pl->fxy + pl->fxy_off[g],
                                    pl->fxyf + pl->fxy_off[g], pl->helmsmem, c.st);
            }));
        }
        IBF_TRY(for_chunks(c, "viscous_x_inverse", cin.data(), nullptr, [&](const UserPtrs &p, int nb) {
            return launch_xinv(mixed, IM_STORE, w, p, 1, 0, nb, pl->xsmem, c.st);
        }));
        for (int g = 0; g < pl->ngrids; ++g) {
            const GridDev &d = pl->grids[g].d;
            double *o = comp == 0 ? out[g].u : (comp == 1 ? out[g].v : out[g].w);
            IBF_TRY(timed(c, "viscous_z", [&]() {
                return launch_zhelm(mixed, w, g, (long long)d.nx * d.ny, comp == 2, pl->helm, pl->helmf, o, c.st);
            }));
        }
    }
    pl->last_stream = c.st;
    return IBF_OK;
}

ibf_status ibf_plan_sync_status(ibf_plan *plan) {
    if (!plan) return IBF_ERR_INVALID_ARG;
    cudaError_t e = cudaSetDevice(plan->device);
    if (e == cudaSuccess) e = cudaStreamSynchronize(plan->last_stream);
    if (e != cudaSuccess) return cuda_fail(e, "cudaStreamSynchronize");
    unsigned word = 0;
    e = cudaMemcpy(&word, plan->work.err, sizeof(word), cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) e = cudaMemset(plan->work.err, 0, sizeof(unsigned));
    if (e != cudaSuccess) return cuda_fail(e, "cudaMemcpy");
    if (word & (1u << IBF_ERR_TIMEOUT)) return IBF_ERR_TIMEOUT;
    if (word & (1u << IBF_ERR_NONFINITE)) return IBF_ERR_NONFINITE;
    if (word & (1u << IBF_WARN_INCOMPATIBLE_RHS)) return IBF_WARN_INCOMPATIBLE_RHS;
    return IBF_OK;
}

ibf_status ibf_plan_destroy(ibf_plan *plan) {
    if (!plan) return IBF_OK;
    cudaSetDevice(plan->device);
    cudaDeviceSynchronize();
    free_all(plan);
    delete plan;
    return IBF_OK;
}

ibf_status ibf_plan_get_info(const ibf_plan *plan, ibf_plan_info *info) {
    if (!plan || !info) return IBF_ERR_INVALID_ARG;
    info->workspace_bytes = plan->ws_bytes;
    info->ngrids = plan->ngrids;
    info->precision = plan->opts.precision;
    info->refine_steps = plan->opts.refine_steps;
    info->total_cells = plan->total_cells;
    return IBF_OK;
}

ibf_status ibf_profile_enable(ibf_plan *plan, int enable) {
    if (!plan) return IBF_ERR_INVALID_ARG;
    plan->prof = enable != 0;
    return IBF_OK;
}

static void prof_collect(ibf_plan *plan) {
    if (plan->prof_pending.empty()) return;
    cudaSetDevice(plan->device);
    cudaEventSynchronize(plan->prof_pending.back().e1);
    for (auto &r : plan->prof_pending) {
        float ms = 0.f;
        cudaEventElapsedTime(&ms, r.e0, r.e1);
        bool found = false;
        for (auto &a : plan->prof_acc)
            if (strcmp(a.first, r.name) == 0) { a.second.first += 1; a.second.second += ms; found = true; break; }
        if (!found) plan->prof_acc.push_back({r.name, {1, (double)ms}});
        plan->ev_pool.push_back(r.e0);
        plan->ev_pool.push_back(r.e1);
    }
    plan->prof_pending.clear();
}

int ibf_profile_read(ibf_plan *plan, const char **names, long long *launches, double *ms, int cap) {
    if (!plan) return 0;
    prof_collect(plan);
    int n = 0;
    for (auto &a : plan->prof_acc) {
        if (n >= cap) break;
        if (names) names[n] = a.first;
        if (launches) launches[n] = a.second.first;
        if (ms) ms[n] = a.second.second;
        ++n;
    }
    return n;
}

ibf_status ibf_profile_reset(ibf_plan *plan) {
    if (!plan) return IBF_ERR_INVALID_ARG;
    prof_collect(plan);
    plan->prof_acc.clear();
    return IBF_OK;
}

}  // extern "C"

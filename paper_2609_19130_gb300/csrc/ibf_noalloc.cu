// ibf_noalloc.cu -- ibf_project_noalloc: the projection of one grid with no device
// allocation at all.
//
// Who needs it: callers that are not allowed to call cudaMalloc (or anything that
// allocates) when they project, for example a host framework whose own allocator owns
// all device memory, code that runs inside a region where an allocation would
// synchronise the device or is forbidden, or real-time loops that must not pay for
// an allocation.  ibf_projection_plan allocates its workspace; this entry point
// instead carves the same workspace out of one fixed, file-scope device array.
//
// The array (kScratchBytes, 64 MiB) exists once per GPU that loads this library and
// stays allocated until the process exits.  Every call uses the same array and
// leaves its contents behind, so two calls that overlap on the GPU (different
// streams, or different host threads) race and corrupt each other: callers must
// order them.  The first call on a device looks up the array's device address
// (cudaGetSymbolAddress) and caches it; that first call should come before any
// stream capture.  Grids whose workspace does not fit are rejected with
// IBF_ERR_UNSUPPORTED_SIZE before anything is launched.
//
// The small per-call tables (grid descriptor, z metrics, twiddles) are built on the
// host and reach the array as the by-value arguments of a copy kernel, in chunks: the
// launch copies the arguments, so no host buffer is read after the call returns and
// no copy from pageable memory waits on the stream.
#include "../../include/ibf.h"

#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <mutex>
#include <vector>

#include "ibf_internal.h"

using namespace ibf;

namespace {

constexpr size_t kScratchBytes = IBF_NOALLOC_SCRATCH_BYTES;
static __device__ __align__(256) unsigned char g_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
void *g_scratch_addr[kMaxDevices] = {nullptr};
std::mutex g_scratch_mu;

// device address of g_scratch on the current device (host code must not use the
// symbol's name as an address)
ibf_status scratch_base(int dev, unsigned char **out) {
    if (dev < 0 || dev >= kMaxDevices) return IBF_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lk(g_scratch_mu);
    if (!g_scratch_addr[dev]) {
        void *p = nullptr;
        if (cudaGetSymbolAddress(&p, g_scratch) != cudaSuccess || !p) {
            (void)cudaGetLastError();
            return IBF_ERR_CUDA;
        }
        g_scratch_addr[dev] = p;
    }
    *out = static_cast<unsigned char *>(g_scratch_addr[dev]);
    return IBF_OK;
}

const int kSizes[] = {1, 2, 3, 4, 6, 8, 12, 16, 24, 32};
bool is_size(int n) {
    for (int s : kSizes)
        if (s == n) return true;
    return false;
}
bool split(int n, int *n1, int *n2) {  // n = n1 n2, n1 >= n2, both register-DFT sizes, balanced
    int b1 = -1, b2 = -1;
    for (int a : kSizes) {
        if (n % a || !is_size(n / a) || a < n / a) continue;
        if (b1 < 0 || a < b1) { b1 = a; b2 = n / a; }
    }
    if (b1 < 0) return false;
    *n1 = b1;
    *n2 = b2;
    return true;
}
FDiv fdiv_of(unsigned d) {
    FDiv f;
    f.d = d;
    unsigned s = 0;
    while ((1ull << s) < d) ++s;
    f.s = s;
    f.m = (unsigned)((((1ull << 32) * ((1ull << s) - d)) / d) + 1);
    return f;
}

// bump allocator over a byte range (offsets only; 256-byte aligned pieces)
struct Carve {
    size_t off = 0;
    size_t take(size_t bytes) {
        const size_t o = off;
        off += (std::max<size_t>(bytes, 16) + 255) & ~(size_t)255;
        return o;
    }
};

// Host-to-device transfer of the per-call tables through kernel arguments: one launch
// per chunk of up to kPutBytes (the chunk travels in the launch's parameter block, which
// sm_70 and newer accept up to 32764 bytes).
constexpr unsigned kPutBytes = 16384;
struct PutChunk {
    uint4 v[kPutBytes / 16];
};
__global__ void __launch_bounds__(256) k_put_chunk(uint4 *dst, unsigned n16, const PutChunk c) {
    for (unsigned i = threadIdx.x; i < n16; i += blockDim.x) dst[i] = c.v[i];
}

}  // namespace

extern "C" ibf_status ibf_project_noalloc(const ibf_grid *grid, const ibf_opts *opts, const ibf_fields *in,
                                          const ibf_fields *out, double dt, double alpha, void *stream) {
    if (!grid || !opts || !in || !out) return IBF_ERR_INVALID_ARG;
    if (!in->u || !in->v || !in->w || !out->u || !out->v || !out->w || !out->p) return IBF_ERR_INVALID_ARG;
    if (in->q) return IBF_ERR_INVALID_ARG;  // no mass source on this entry point
    if (!(dt > 0) || !(alpha > 0) || !std::isfinite(dt) || !std::isfinite(alpha)) return IBF_ERR_INVALID_ARG;
    if (opts->precision != IBF_FP64 && opts->precision != IBF_MIXED) return IBF_ERR_INVALID_ARG;
    if (opts->refine_steps < 0 || opts->refine_steps > 8 || opts->pressure != IBF_P_PHI) return IBF_ERR_INVALID_ARG;
    if (opts->precision == IBF_FP64 && opts->refine_steps != 0) return IBF_ERR_INVALID_ARG;
    const ibf_grid &g = *grid;
    // the checks of ibf_projection_plan (sizes, lengths, faces or tanh factor, boundary
    // conditions), then the restrictions of this entry point
    std::vector<double> zf;
    {
        const ibf_status vs = validate_grid(grid, zf);
        if (vs != IBF_OK) return vs;
    }
    if (g.bc_x != IBF_BC_PERIODIC || g.bc_y != IBF_BC_PERIODIC || g.bc_zlo != IBF_BC_NEUMANN ||
        g.bc_zhi != IBF_BC_NEUMANN)
        return IBF_ERR_UNSUPPORTED_BC;
    GridDev d;
    memset(&d, 0, sizeof(d));
    if (!split(g.nx, &d.nx1, &d.nx2) || !split(g.ny, &d.ny1, &d.ny2)) return IBF_ERR_UNSUPPORTED_SIZE;
    const int mixed = opts->precision == IBF_MIXED;
    const int nz = g.nz;

    int dev = 0, nsm = 0, optin = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess) {
        (void)cudaGetLastError();
        return IBF_ERR_CUDA;
    }
    const size_t csz = mixed ? 8 : 16, rsz = mixed ? 4 : 8;

    // launch shapes: the rules of ibf_projection_plan for a one-grid plan
    d.nx = g.nx; d.ny = g.ny; d.nz = nz;
    d.nxh = d.nx / 2 + 1;
    d.nxu = d.nx;  // periodic x and y only: no wall faces
    d.nyv = d.ny;
    const int mbmax = std::max(1, std::min(d.nxh, 4096 / d.ny));
    const int want = (64 + d.ny2 - 1) / d.ny2;
    const int slots = (mixed ? kYZResidentF32 : kYZResidentF64) * nsm;  // the rule of ibf_projection_plan
    d.mb = std::min(std::min(mbmax, want), std::max(1, (d.nxh + slots - 1) / slots));
    d.ncb = (d.nxh + d.mb - 1) / d.mb;
    int rows = 2 * std::max(1, (mixed ? 8192 : 4096) / d.nx);
    rows = std::min(rows, (d.ny + 1) & ~1);
    d.rows = std::max(2, rows);
    d.nrb = (d.ny + d.rows - 1) / d.rows;
    d.dx = g.lx / d.nx; d.dy = g.ly / d.ny;
    d.rdx = 1.0 / d.dx; d.rdy = 1.0 / d.dy;
    d.inv_nxy = 1.0 / ((double)d.nx * d.ny);
    d.sum_hz = g.lz;
    d.fnx = fdiv_of(d.nx); d.fnx1 = fdiv_of(d.nx1); d.fnx2 = fdiv_of(d.nx2);
    d.fnph = fdiv_of(d.nx / 2 + 1);
    d.fny1 = fdiv_of(d.ny1); d.fny2 = fdiv_of(d.ny2);
    d.fmb = fdiv_of(d.mb); d.frows = fdiv_of(d.rows); d.fnpair = fdiv_of(d.rows / 2);
    d.fnpair2 = fdiv_of(d.rows / 4 > 0 ? d.rows / 4 : 1);
    const size_t cells = (size_t)d.nx * d.ny * nz;
    const size_t nspec = (size_t)nz * d.ncb * d.ny * d.mb;
    const size_t xsmem = (size_t)(d.rows / 2) * (size_t)(d.nx1 * (d.nx2 + 1) + 1) * csz;
    size_t yzsmem;
    {
        const size_t sstr = (size_t)(d.ny1 * (d.ny2 + 1) + 1), nslot = (size_t)d.ny * d.mb;
        const size_t fwd = kYZStages * ((d.mb * sstr * csz + nslot * rsz + 15) & ~(size_t)15) + nslot * csz;
        const size_t bwd = kYZStages * ((nslot * (csz + rsz) + 15) & ~(size_t)15) + (d.mb * sstr + nslot) * csz;
        yzsmem = std::max(fwd, bwd);
        if (mixed && d.mb == 1 && !d.wall_y)
            yzsmem = std::max(yzsmem, std::max(yz_pipe_smem(d.ny, (int)sstr), yz_bulk_smem(d.ny, (int)sstr)));
    }
    const size_t smem00 = (size_t)10 * (nz + 1) * 8;
    const size_t cap = smem_cap_of(optin);  // the limit ibf_projection_plan applies
    if (xsmem > cap || yzsmem > cap || smem00 > cap) return IBF_ERR_UNSUPPORTED_SIZE;

    // layout inside the scratch array: first the small tables uploaded from the host
    // (one copy), then the workspace written by the kernels
    Carve cv;
    const size_t o_grid = cv.take(sizeof(GridDev));
    const size_t o_xs = cv.take(2 * sizeof(int)), o_ys = cv.take(2 * sizeof(int)), o_slab = cv.take(2 * sizeof(int));
    const size_t L = (size_t)nz + 1;
    const size_t o_hz = cv.take(L * 8), o_rhz = cv.take(L * 8), o_rgzf = cv.take(L * 8), o_az = cv.take(L * 8),
                 o_cz = cv.take(L * 8), o_inv00 = cv.take(L * 8), o_azf = cv.take(L * 4), o_czf = cv.take(L * 4),
                 o_rhzdf = cv.take(L * 8), o_rgzfdf = cv.take(L * 8);
    const size_t o_twx = cv.take(csz * 2 * d.nx), o_twy = cv.take(csz * 2 * d.ny);
    const size_t upload_bytes = cv.off;
    const size_t o_spec = cv.take(csz * nspec), o_tab = cv.take(rsz * nspec);
    const size_t o_bdf = mixed ? cv.take(8 * cells) : 0;
    const size_t o_phh = mixed ? cv.take(4 * cells) : 0, o_phl = mixed ? cv.take(4 * cells) : 0;
    const int R = mixed ? opts->refine_steps : 0;
    const size_t o_phl2 = (mixed && R >= 2) ? cv.take(4 * cells) : 0;
    const size_t npart = (size_t)nz * d.nrb;  // no half-block forward x-FFT CTAs here
    const size_t o_part = cv.take(8 * npart), o_partp = cv.take(8 * npart);
    const size_t o_mean = cv.take(8), o_maxb = cv.take(8), o_maxd = cv.take(8), o_err = cv.take(4);
    const size_t o_sol00 = cv.take(8 * L);
    if (cv.off > kScratchBytes) return IBF_ERR_UNSUPPORTED_SIZE;

    unsigned char *base = nullptr;
    ibf_status s = scratch_base(dev, &base);
    if (s != IBF_OK) return s;

    // host image of the uploaded part
    std::vector<unsigned char> img(upload_bytes, 0);
    auto put = [&](size_t o, const void *src, size_t n) { memcpy(img.data() + o, src, n); };
    d.spec_off = 0; d.cell_off = 0; d.tab_off = 0; d.z_off = 0; d.part_off = 0;
    d.twx_off = 0; d.twy_off = 0; d.xblk_off = 0; d.yzblk_off = 0;
    put(o_grid, &d, sizeof(d));
    const int xs[2] = {0, nz * d.nrb}, ys[2] = {0, d.ncb};
    put(o_xs, xs, sizeof(xs));
    put(o_ys, ys, sizeof(ys));
    const int none[2] = {0, 0};  // streaming y/z kernels only: no resident-slab blocks
    put(o_slab, none, sizeof(none));
    std::vector<double> hz(L, 0.0), rhz(L, 0.0), rgzf(L, 0.0), az(L, 0.0), cz(L, 0.0), inv00(L, 0.0);
    std::vector<float> azf(L), czf(L), rhzdf(2 * L), rgzfdf(2 * L);
    for (int k = 0; k < nz; ++k) { hz[k] = zf[k + 1] - zf[k]; rhz[k] = 1.0 / hz[k]; }
    for (int k = 1; k < nz; ++k) rgzf[k] = 1.0 / (0.5 * (zf[k] + zf[k + 1]) - 0.5 * (zf[k - 1] + zf[k]));
    for (int k = 0; k < nz; ++k) { az[k] = rhz[k] * rgzf[k]; cz[k] = rhz[k] * rgzf[k + 1]; }
    double cp = 0.0;
    for (int k = 1; k < nz; ++k) {
        inv00[k] = 1.0 / (-(az[k] + cz[k]) - az[k] * cp);
        cp = cz[k] * inv00[k];
    }
    for (size_t k = 0; k < L; ++k) {
        azf[k] = (float)az[k];
        czf[k] = (float)cz[k];
        float h = (float)rhz[k];
        rhzdf[2 * k] = h; rhzdf[2 * k + 1] = (float)(rhz[k] - (double)h);
        h = (float)rgzf[k];
        rgzfdf[2 * k] = h; rgzfdf[2 * k + 1] = (float)(rgzf[k] - (double)h);
    }
    put(o_hz, hz.data(), L * 8); put(o_rhz, rhz.data(), L * 8); put(o_rgzf, rgzf.data(), L * 8);
    put(o_az, az.data(), L * 8); put(o_cz, cz.data(), L * 8); put(o_inv00, inv00.data(), L * 8);
    put(o_azf, azf.data(), L * 4); put(o_czf, czf.data(), L * 4);
    put(o_rhzdf, rhzdf.data(), L * 8); put(o_rgzfdf, rgzfdf.data(), L * 8);
    // four-step twiddles w^(a b), w = exp(-2 pi i / n), in the solve precision: forward
    // table F[q n2 + c] = w^(q c), then inverse table I[p n1 + q1] = w^(p q1)
    auto tw = [&](size_t o, int n, int n1) {
        const int n2 = n / n1;
        auto one = [&](size_t i, long long e) {
            const double a = 2.0 * M_PI * (double)(e % n) / (double)n, c = std::cos(a), sn = -std::sin(a);
            if (mixed) { const float v[2] = {(float)c, (float)sn}; put(o + 8 * i, v, 8); }
            else { const double v[2] = {c, sn}; put(o + 16 * i, v, 16); }
        };
        for (int q = 0; q < n1; ++q)
            for (int c = 0; c < n2; ++c) one((size_t)q * n2 + c, (long long)q * c);
        for (int p = 0; p < n2; ++p)
            for (int q1 = 0; q1 < n1; ++q1) one((size_t)n + (size_t)p * n1 + q1, (long long)p * q1);
    };
    tw(o_twx, d.nx, d.nx1);
    tw(o_twy, d.ny, d.ny1);

    cudaStream_t st = static_cast<cudaStream_t>(stream);
    // the tables, chunk by chunk, as kernel arguments (upload_bytes is a multiple of 256)
    for (size_t o = 0; o < upload_bytes; o += kPutBytes) {
        const size_t n = std::min<size_t>(kPutBytes, upload_bytes - o);
        PutChunk c;
        memcpy(c.v, img.data() + o, n);
        k_put_chunk<<<1, 256, 0, st>>>(reinterpret_cast<uint4 *>(base + o), (unsigned)(n / 16), c);
        if (cudaGetLastError() != cudaSuccess) return IBF_ERR_CUDA;
    }
    if (cudaMemsetAsync(base + o_err, 0, 4, st) != cudaSuccess) return IBF_ERR_CUDA;

    Work w;
    memset(&w, 0, sizeof(w));
    w.grids = reinterpret_cast<const GridDev *>(base + o_grid);
    w.ngrids = 1;
    w.xblk_start = reinterpret_cast<const int *>(base + o_xs);
    w.yzblk_start = reinterpret_cast<const int *>(base + o_ys);
    w.ystr_start = w.yzblk_start;
    w.slab_start = reinterpret_cast<const int *>(base + o_slab);
    w.yfft_start = w.slab_start;  // no split-path blocks either
    w.sweep_start = w.slab_start;
    w.sol00 = reinterpret_cast<double *>(base + o_sol00);
    w.z.hz = reinterpret_cast<double *>(base + o_hz);
    w.z.rhz = reinterpret_cast<double *>(base + o_rhz);
    w.z.rgzf = reinterpret_cast<double *>(base + o_rgzf);
    w.z.az = reinterpret_cast<double *>(base + o_az);
    w.z.cz = reinterpret_cast<double *>(base + o_cz);
    w.z.inv00 = reinterpret_cast<double *>(base + o_inv00);
    w.z.azf = reinterpret_cast<float *>(base + o_azf);
    w.z.czf = reinterpret_cast<float *>(base + o_czf);
    w.z.rhz_df = reinterpret_cast<float2 *>(base + o_rhzdf);
    w.z.rgzf_df = reinterpret_cast<float2 *>(base + o_rgzfdf);
    w.spec = base + o_spec;
    w.tab = base + o_tab;
    w.twx = base + o_twx;
    w.twy = base + o_twy;
    if (mixed) {
        w.bdf = reinterpret_cast<float2 *>(base + o_bdf);
        w.phi_hi = reinterpret_cast<float *>(base + o_phh);
        w.phi_lo = reinterpret_cast<float *>(base + o_phl);
        if (R >= 2) w.phi_lo2 = reinterpret_cast<float *>(base + o_phl2);
    }
    w.partial = reinterpret_cast<double *>(base + o_part);
    w.partial_phi = reinterpret_cast<double *>(base + o_partp);
    w.mean_b = reinterpret_cast<double *>(base + o_mean);
    w.maxb = reinterpret_cast<unsigned long long *>(base + o_maxb);
    w.maxdiv = reinterpret_cast<unsigned long long *>(base + o_maxd);
    w.err = reinterpret_cast<unsigned *>(base + o_err);

    UserPtrs p;
    memset(&p, 0, sizeof(p));
    p.in_u[0] = in->u; p.in_v[0] = in->v; p.in_w[0] = in->w;
    p.out_u[0] = out->u; p.out_v[0] = out->v; p.out_w[0] = out->w; p.out_p[0] = out->p;
    p.g0 = 0; p.g1 = 1; p.blk0 = 0;

    const int nxblk = nz * d.nrb, nyz = d.ncb;
    const double sc = alpha * dt, rs = 1.0 / sc;
    cudaError_t e = set_smem_limits(mixed);
    if (e == cudaSuccess) e = launch_build_table(mixed, w, nyz, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(base + o_maxb, 0, 16, st);
    if (e == cudaSuccess) e = launch_xfwd(mixed, XM_DIV, w, p, 0, 0, nxblk, sc, rs, xsmem, st);
    auto solve = [&](int first) {
        cudaError_t r = launch_yzfwd(mixed, w, nyz, yzsmem, st);
        if (r == cudaSuccess) r = launch_k00(w, mixed, first, nz, st);
        if (r == cudaSuccess) r = launch_yzbwd(mixed, w, nyz, yzsmem, st);
        return r;
    };
    if (e == cudaSuccess) e = solve(1);
    if (e == cudaSuccess) e = launch_xinv(mixed, IM_STORE, w, p, 0, 0, nxblk, xsmem, st);
    // the refinement sweeps as in ibf_project: the last of two or more keeps its
    // correction apart in phi_lo2
    for (int r = 0; r < R && e == cudaSuccess; ++r) {
        e = launch_xfwd(mixed, XM_RESID, w, p, 0, r > 0, nxblk, sc, rs, xsmem, st);
        if (e == cudaSuccess) e = solve(0);
        const int im = (R >= 2 && r == R - 1) ? IM_LAST : IM_ACCUM;
        if (e == cudaSuccess) e = launch_xinv(mixed, im, w, p, 0, r > 0, nxblk, xsmem, st);
    }
    if (e == cudaSuccess) e = launch_correct(mixed, 0, w, p, 0, R > 0, R >= 2, nxblk, sc, IBF_P_PHI, 0.0, st);
    if (e != cudaSuccess) {
        (void)cudaGetLastError();
        return IBF_ERR_CUDA;
    }
    return IBF_OK;
}

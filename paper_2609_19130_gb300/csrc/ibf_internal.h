// ibf_internal.h -- plan-internal data shared by the host plan code (ibf_capi.cpp)
// and the kernels (ibf_kernels.cu).  Not part of the public ABI.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <vector>

#include "../../include/ibf.h"

namespace ibf {

// Largest number of grids whose user pointers travel in one launch's parameters.
constexpr int kGridsPerLaunch = 32;
// Thread counts of the kernels.
constexpr int kXThreads = 256;   // x-direction (row) kernels and stencil kernels
constexpr int kYZThreads = 128;  // y-FFT + z-tridiagonal column kernels
constexpr int kYZStages = 2;     // planes in flight per column block in the yz kernels
// CTAs of the streaming y/z kernels resident per SM (registers: fp32 kernels are capped at
// 128 registers per thread; the fp64 ones use about 255)
constexpr int kYZResidentF32 = 4, kYZResidentF64 = 2;
// Pipelined streaming y/z kernels (mixed path, one x-mode per column block, periodic y):
// ring entries of FFT buffers (and pivot chunks) in shared memory
constexpr int kPipeF = 3;  // forward: [FFT buffer | pivots] for the planes being copied, transformed, swept
constexpr int kPipeB = 4;  // backward: FFT buffers being copied, swept, transformed, stored (pivots: 2)
__host__ __device__ inline size_t pipe_align16(size_t b) { return (b + 15) & ~(size_t)15; }
// shared memory of the pipelined kernels; sstr = padded FFT sequence length (complex)
inline size_t yz_pipe_smem(int ny, int sstr) {
    const size_t fwd = kPipeF * pipe_align16((size_t)sstr * 8 + (size_t)ny * 4) + (size_t)ny * 8;
    const size_t bwd = kPipeB * pipe_align16((size_t)sstr * 8) + 2 * pipe_align16((size_t)ny * 4) + (size_t)ny * 8;
    return fwd > bwd ? fwd : bwd;
}
// Round-based pipelined y/z kernels (same launch; even ny): kBulkPlanes planes per round,
// one FFT warp each, copied as whole planes with bulk asynchronous copies into two sets
// of buffers (the next round's planes arrive while this round is computed)
constexpr int kBulkPlanes = 3;
constexpr unsigned kBulkWaitLimit = 1u << 20;  // polls of an mbarrier before a copy counts as lost
inline size_t yz_bulk_smem(int ny, int sstr) {
    const size_t sb = pipe_align16((size_t)sstr * 8 > (size_t)ny * 8 ? (size_t)sstr * 8 : (size_t)ny * 8);
    return 2 * kBulkPlanes * sb + 2 * kBulkPlanes * 8;
}
constexpr int kSlabThreads = 256;  // resident-slab y/z kernel
constexpr int kSweepThreads = 256; // split y/z path: Thomas sweeps, one thread per mode
// spectral z: z lines (slots of a plane) per k_zdct CTA, mixed / fp64
constexpr int kZdctLinesF32 = 16, kZdctLinesF64 = 8;

// Division by a run-time invariant d (Granlund & Montgomery, PLDI 1994, round-up
// variant): n / d = (umulhi(n, m) + n) >> s for 0 <= n < 2^31.
struct FDiv {
    unsigned d, m, s;
};

// Per-grid descriptor, one entry per grid in device memory.
struct GridDev {
    int nx, ny, nz, nxh;       // cells; x-modes kept: nx/2 + 1 (real FFT) or nx (DCT-II)
    int wall_x, wall_y;        // 1: that direction is wall-bounded (Neumann phi, DCT-II transform)
    int nxu, nyv;              // faces of u per row (nx + wall_x), rows of v per plane (ny + wall_y)
    int dctx_off, dcty_off;    // offsets of the exp(-i pi m/(2N)) tables of the DCTs (in twx / twy)
    int dir_top;               // 1: homogeneous Dirichlet phi on the top face (outlet), else Neumann
    double ez_top;             // Dirichlet outlet: extra diagonal of level nz-1, rhz / (lz - zc_{nz-1})
    int yzk;                   // y/z kernels: 0 streaming (k_yzfwd + k_yzbwd), 1 resident slab (k_yzslab),
                               // 2 split (k_yfft, k_zsweep_fwd / k_zsweep_bwd), 3 spectral z (k_yfft,
                               // k_zdct: DCT along z, uniform z with Neumann walls)
    int nz1, nz2;              // spectral z: two-level FFT factors of nz
    int twz_off, dctz_off;     // spectral z: four-step and DCT twiddles of nz (in twy)
    int cr_levels;             // slab kernel: cyclic-reduction levels before Thomas (0: Thomas with the table)
    int nx1, nx2, ny1, ny2;    // two-level FFT factors: nx = nx1*nx2, ny = ny1*ny2
    int mb, ncb;               // x-modes per column block of the yz kernels, number of blocks
    int rows, nrb;             // rows per CTA of the x kernels (even), row blocks per plane
    long long spec_off;        // offset of the grid's spectrum (complex elements)
    long long cell_off;        // offset of the grid's per-cell workspace (cells)
    long long tab_off;         // offset of the grid's pivot table (entries)
    int z_off;                 // offset of the grid's per-level arrays ((nz+1) entries each)
    int part_off;              // offset of the grid's partial sums (nz * nrb entries, twice that with xfwd_split)
    int twx_off, twy_off;      // offsets of exp(-2 pi i r/N) tables for nx and ny (complex entries)
    int xblk_off, yzblk_off;   // first block of the grid in x-kernel / yz-kernel launches
    double dx, dy, rdx, rdy;   // spacings and their inverses
    double inv_nxy;            // 1 / (nx ny)
    double sum_hz;             // lz
    FDiv fnx, fnx1, fnx2, fny1, fny2, fmb, frows, fnpair, fnph;  // fnph: nx/2 + 1
    FDiv fnpair2;              // rows / 4 (row pairs of the half-block CTAs of the inverse x-FFT)
    FDiv fnz1, fnz2;           // spectral z: nz1, nz2
};

// Per-level arrays (index z_off + k; nz+1 entries per grid, the last one only used where noted).
struct ZArrays {
    double *hz;      // hz_k (k < nz)
    double *rhz;     // 1/hz_k
    double *rgzf;    // 1/gz_k on interior faces 1..nz-1, 0 on the wall faces 0 and nz (nz+1 entries)
    double *az, *cz; // tridiagonal off-diagonals: az_k = rhz_k rgzf_k, cz_k = rhz_k rgzf_{k+1}
    double *inv00;   // pivots of the pinned (0,0) system (inv00_0 = 0)
    float *azf, *czf;        // fp32 copies of az, cz
    float2 *rhz_df, *rgzf_df; // float-float copies (hi, lo) of rhz, rgzf
};

// Workspace pointers of a plan, passed by value to the kernels.
struct Work {
    const GridDev *grids;      // [ngrids]
    int ngrids;
    int walls;                 // some grid has a wall-bounded x or y (selects the kernels that handle it)
    int xinv_split;            // mixed path, every grid's rows divisible by 4: half-block inverse x-FFT CTAs
    int xfwd_split;            // the same condition: half-block forward x-FFT CTAs
    const int *xblk_start;     // prefix of x-kernel blocks over grids [ngrids+1]
    const int *yzblk_start;    // prefix of column blocks over all grids [ngrids+1] (pivot table)
    const int *ystr_start;     // prefix of column blocks over grids with streaming y/z kernels
    const int *slab_start;     // prefix of column blocks over grids with the resident-slab kernel
    const int *yfft_start;     // split path: prefix of (plane, column block) FFT blocks over grids
    const int *sweep_start;    // split path: prefix of Thomas-sweep blocks (kSweepThreads modes each)
    const int *zdct_start;     // spectral z: prefix of k_zdct blocks (zdct_lines(T) z lines each)
    double *sol00;             // per level (z_off + k): solution of the (0,0) mode, written by k_00
    ZArrays z;
    void *spec;                // complex<T> spectrum, per grid nz*ncb*ny*mb
    void *tab;                 // T pivot table, same layout as spec (real entries)
    const void *twx, *twy;     // complex<T> twiddle tables
    float2 *bdf;               // float-float right-hand side (mixed path) per cell
    double *phi_ws;            // per-cell fp64 phi of the adjoint solve / of a pressure update (fp64 path)
    double *bws;               // per-cell fp64 right-hand side (fp64 path with the implicit pressure update)
    float *phi_hi, *phi_lo;    // per-cell float-float phi being refined (mixed path)
    float2 *rdf;               // per-cell float-float residual of the first refinement sweep (mixed path
                               // with two or more sweeps; else null): the second sweep's starts from it
    float *phi_lo2;            // per-cell correction of the last refinement sweep, kept apart so that
                               // phi = hi + lo + lo2 carries more bits than a float-float pair
                               // (mixed path with two or more sweeps; else null)
    double *partial;           // per (grid, k, row block, half with xfwd_split) plane sums of the right-hand side
    double *partial_phi;       // the same of the current phi (refinement)
    double *mean_b;            // [ngrids] removed weighted mean of the first right-hand side
    unsigned long long *maxb;  // [ngrids] max |rhs| (double bits), for max|D u*|
    unsigned long long *maxdiv;// [ngrids] max |D u| of the output (double bits)
    unsigned *err;             // device error word (bit i: ibf_status i)
    int fault_lose_copy;       // test hook (IBF_FAULT_LOSE_COPY): the round-based forward y/z kernel
                               // skips one plane copy, so that its bounded wait runs out
};

// Per-launch user pointers for up to kGridsPerLaunch grids.
struct UserPtrs {
    const double *in_u[kGridsPerLaunch], *in_v[kGridsPerLaunch], *in_w[kGridsPerLaunch], *in_p[kGridsPerLaunch];
    double *out_u[kGridsPerLaunch], *out_v[kGridsPerLaunch], *out_w[kGridsPerLaunch], *out_p[kGridsPerLaunch];
    const double *in_q[kGridsPerLaunch];  // mass sources of Eq. (elliptic) (may be null)
    int g0, g1;                // grids [g0, g1) of this launch
    int blk0;                  // first block index (x-kernel numbering) of grid g0
    int zshift;                // XM_COPY: plane k of the transform reads plane k + zshift of in_u
                               // (1: interior z-faces of w; the last plane is then zero)
};

// x-forward modes: right-hand side of the first solve, refinement residual (phi a
// float-float pair), adjoint source, refinement residual of the first sweep (phi plain fp32)
enum XMode { XM_DIV = 0, XM_RESID = 1, XM_ADJ = 2, XM_RESID0 = 3, XM_DIVQ = 4 /* XM_DIV with a mass source q */,
             XM_COPY = 5 /* the field in_u itself (viscous solve): no stencil, no plane sums */,
             XM_RESID1 = 6 /* second sweep: the first sweep's residual less L of its correction */ };
enum InvMode { IM_STORE = 0, IM_ACCUM = 1, IM_LAST = 2 /* the last sweep's correction into phi_lo2 */ };

// Launchers (ibf_kernels.cu).  T = 0: fp64 path, 1: mixed path.
cudaError_t launch_xfwd(int mixed, int mode, const Work &w, const UserPtrs &p, int use_ws, int lo_valid, int nblk,
                        double s, double rs, size_t smem, cudaStream_t st);
cudaError_t launch_yzfwd(int mixed, const Work &w, int nblk, size_t smem, cudaStream_t st);
cudaError_t launch_yzbwd(int mixed, const Work &w, int nblk, size_t smem, cudaStream_t st);
cudaError_t launch_k00(const Work &w, int mixed, int first_solve, int maxnz, cudaStream_t st);
cudaError_t launch_yzslab(int mixed, const Work &w, int nblk, size_t smem, cudaStream_t st);
cudaError_t launch_yfft(int mixed, int inverse, const Work &w, int nblk, size_t smem, cudaStream_t st);
cudaError_t launch_zsweep(int mixed, int backward, const Work &w, int nblk, cudaStream_t st);
cudaError_t launch_zdct(int mixed, const Work &w, int nblk, size_t smem, cudaStream_t st);
cudaError_t launch_xinv(int mixed, int mode, const Work &w, const UserPtrs &p, int use_ws, int lo_valid, int nblk,
                        size_t smem, cudaStream_t st);
// lo2: phi is hi + lo + lo2 (the last sweep's correction in phi_lo2; mixed path, two or more sweeps)
cudaError_t launch_correct(int mixed, int adjoint, const Work &w, const UserPtrs &p, int use_ws, int lo_valid,
                           int lo2, int nblk, double s, int pmode, double cimp, cudaStream_t st);
cudaError_t launch_divstat(int mixed, const Work &w, const UserPtrs &p, int nblk, cudaStream_t st);
cudaError_t launch_finalize(const Work &w, double *max_div, double *max_div_in, double *compat, double s,
                            cudaStream_t st);
cudaError_t launch_build_table(int mixed, const Work &w, int nblk, cudaStream_t st);
cudaError_t set_smem_limits(int mixed);
cudaError_t set_smem_limits_yz(int mixed);  // the y/z kernels' share of set_smem_limits
cudaError_t set_smem_cap(const void *fn);   // one kernel's dynamic shared-memory cap

// Host side (ibf_capi.cpp), shared by the plan and the no-allocation entry point.
// Validates one grid descriptor and fills zf with its nz + 1 z faces.
ibf_status validate_grid(const ibf_grid *g, std::vector<double> &zf);
// Dynamic shared memory a plan lets one kernel request: the device's opt-in maximum
// per block less a margin for the kernels' static shared memory.
inline size_t smem_cap_of(int optin_bytes) { return (size_t)optin_bytes - 1024; }

}  // namespace ibf

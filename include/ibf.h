/*
 * ibf.h -- C ABI of the GB300 pressure-projection library (libibf.so).
 *
 * The library computes the projection step of the fractional-step
 * Navier-Stokes solver of IB-Flows (Section "Fluid Mechanics"):
 *
 *   Eq. (elliptic):  lap(phi) = div(u*) / (alpha dt)          (q = 0)
 *   Eq. (velsolen):  u_{n+1}  = u* - alpha dt grad(phi)
 *
 * on the staggered Cartesian grid with second-order centred differences, x and
 * y periodic with uniform spacing, z bounded by walls with an arbitrary
 * (stretched) spacing and a homogeneous Neumann condition for phi, the
 * arbitrary constant of phi fixed by a reference value (same section).  The
 * Poisson equation is solved directly as the paper's solver does (Section
 * "Fluid domain", projection paragraph): real FFTs in x and y leave one
 * tridiagonal system along z per horizontal mode.  Everything runs on one GPU
 * in hand-written sm_103a kernels; there is no CPU fallback.
 *
 * Beyond the paper (which has x and y periodic), x and/or y may also be
 * wall-bounded (IBF_BC_NEUMANN): that direction then uses a DCT-II, computed
 * with an FFT of the same length between a reordering and pre/post twiddles
 * (Makhoul 1980), instead of the real FFT.
 *
 * Discretisation fixed by this library (the paper's Section "Fluid Mechanics" gives
 * only the scheme's type, staggered, and its order, second-order centred):
 *   cells i < nx, j < ny, k < nz;  dx = lx/nx, dy = ly/ny;
 *   z faces zf[0..nz] with zf[0] = 0, zf[nz] = lz;  hz_k = zf[k+1]-zf[k];
 *   cell centres zc_k = (zf_k + zf_{k+1})/2;  gz_k = zc_k - zc_{k-1};
 *   u[k][j][i] on the x-face x = i dx (left face of cell i), shape [nz][ny][nx],
 *     or [nz][ny][nx+1] when x is wall-bounded (faces 0 and nx are the walls);
 *   v[k][j][i] on the y-face y = j dy, shape [nz][ny][nx], or [nz][ny+1][nx] when y
 *     is wall-bounded (rows 0 and ny are the walls);
 *   w[k][j][i] on the z-face z = zf[k], shape [nz+1][ny][nx] (k = 0, nz: walls);
 *   p (phi)   at cell centres, shape [nz][ny][nx];  all float64, i fastest.
 *   (D u)_c = (u_{i+1}-u_i)/dx + (v_{j+1}-v_j)/dy + (w_{k+1}-w_k)/hz_k (wrap in a
 *   periodic direction);
 *   G phi on interior faces (difference over dx, dy or gz_k), zero on the walls,
 *   so the wall-normal velocity is left unchanged (a Dirichlet outlet instead takes
 *   -phi_{nz-1} / (lz - zc_{nz-1}) on the top face).
 *   Reference value: the volume-weighted mean of the right-hand side is removed
 *   (its value is reported as the compatibility defect) and phi is returned
 *   with zero volume-weighted mean (weights dx dy hz_k).
 *
 * Threading: a plan may be used by one host thread and one stream at a time.
 * Calls never throw; every entry point returns an ibf_status.
 */
#ifndef IBF_H
#define IBF_H

#ifdef __cplusplus
extern "C" {
#endif

#define IBF_VERSION_MAJOR 0
#define IBF_VERSION_MINOR 1
#define IBF_MAX_GRIDS 4096

typedef enum ibf_status {
    IBF_OK = 0,
    IBF_ERR_INVALID_ARG = 1,      /* null pointer, non-positive size, bad enum, ... */
    IBF_ERR_UNSUPPORTED_SIZE = 2, /* nx or ny not a product of two factors in {1,2,3,4,6,8,12,16,24,32} */
    IBF_ERR_OOM = 3,              /* a device allocation in ibf_projection_plan failed */
    IBF_ERR_CUDA = 4,             /* a CUDA runtime call failed (message: ibf_last_error) */
    IBF_ERR_TIMEOUT = 5,          /* a bounded device wait gave up (reported by ibf_plan_sync_status) */
    IBF_ERR_NONFINITE = 6,        /* NaN or Inf met in the right-hand side (ibf_plan_sync_status) */
    IBF_WARN_INCOMPATIBLE_RHS = 7,/* |compatibility defect| above 1e-8 of the RHS scale; result still returned */
    IBF_ERR_UNSUPPORTED_BC = 8    /* a boundary condition the library does not implement (Dirichlet in
                                     x, y or at the bottom, periodic z; for ibf_project_noalloc also
                                     walls in x or y and a Dirichlet outlet; for ibf_viscous_solve
                                     walls in x or y) */
} ibf_status;

typedef enum ibf_bc {
    IBF_BC_PERIODIC = 0,
    IBF_BC_NEUMANN = 1,           /* wall: prescribed normal velocity, homogeneous Neumann phi */
    IBF_BC_DIRICHLET = 2          /* homogeneous Dirichlet phi: the top (outlet) face only */
} ibf_bc;

/* Output pressure (paper Eq. pressure).  IBF_P_PHI: out.p = phi.  IBF_P_EXPLICIT:
 * out.p = p_n + phi (explicit viscous terms).  IBF_P_IMPLICIT: out.p = p_n + phi -
 * alpha dt / (2 Re) lap(phi) (Crank-Nicolson viscous terms), with lap(phi) taken as
 * the right-hand side the solve satisfies, b - <b> (b = D u* / (alpha dt)), which is
 * the discrete Laplacian of the returned phi up to the solver's residual.  p_n is
 * in[g].p (required for the last two); out.p may alias it. */
typedef enum ibf_pressure {
    IBF_P_PHI = 0,
    IBF_P_EXPLICIT = 1,
    IBF_P_IMPLICIT = 2
} ibf_pressure;

typedef enum ibf_precision {
    IBF_FP64 = 0,  /* fp64 transforms, tridiagonal sweeps and stencils */
    IBF_MIXED = 1  /* fp32 transforms and sweeps; float-float (2 x fp32) stencils, residual and
                      accumulation; refine_steps iterative-refinement sweeps */
} ibf_precision;

/* One grid of the batch.  Copied by ibf_projection_plan; the caller keeps ownership of zf. */
typedef struct ibf_grid {
    int nx, ny, nz;         /* cells; nx, ny as for IBF_ERR_UNSUPPORTED_SIZE, nz >= 1 */
    double lx, ly, lz;      /* box lengths (> 0) */
    const double *zf;       /* HOST pointer to nz+1 strictly ascending z faces with zf[0] = 0 and
                               zf[nz] = lz, or NULL to use the tanh map below */
    double beta;            /* tanh clustering factor when zf == NULL:
                               zf_k = lz/2 (1 + tanh(beta (2k/nz - 1)) / tanh(beta)); beta = 0: uniform */
    int bc_x, bc_y;         /* ibf_bc: IBF_BC_PERIODIC, or IBF_BC_NEUMANN (walls, DCT-II) */
    int bc_zlo, bc_zhi;     /* ibf_bc: bc_zlo IBF_BC_NEUMANN; bc_zhi IBF_BC_NEUMANN, or IBF_BC_DIRICHLET
                               for an outlet (phi = 0 on the top face through the mirror value
                               -phi_{nz-1}; the top face velocity is then corrected, and no
                               compatibility mean or reference value is involved) */
} ibf_grid;

typedef struct ibf_opts {
    int precision;          /* ibf_precision */
    int refine_steps;       /* IBF_MIXED only: iterative-refinement sweeps after the first solve (0..8) */
    int autotune;           /* 1: time candidate launch shapes (ibf_tuning) at plan time, once per
                               distinct grid shape and precision in the process (allocates
                               temporary device buffers, synchronises the device); with the
                               environment variable IBF_AUTOTUNE_LOG set, every timed
                               candidate is printed to stderr */
    int pressure;           /* what out.p receives (Eq. pressure), ibf_pressure; default IBF_P_PHI */
    double inv_re;          /* 1/Re of the implicit viscous term (IBF_P_IMPLICIT; >= 0) */
} ibf_opts;

/* DEVICE pointers (float64, layouts above) of one grid.  q (input only, may be NULL =
 * zero): the cell-centred mass source of Eq. (elliptic), lap(phi) = (D u* - q)/(alpha dt),
 * layout of p; with it the projected velocity satisfies D u = q. */
typedef struct ibf_fields {
    double *u, *v, *w, *p;
    const double *q;
} ibf_fields;

/* Optional DEVICE outputs, each an array of ngrids doubles (any pointer may be NULL).
 * max_div     : max_c |(D u_{n+1} - q)_c| of the returned velocity (q = 0 if absent);
 * max_div_in  : max_c |(D u* - q)_c|;
 * compat      : removed volume-weighted mean of div(u*)/(alpha dt). */
typedef struct ibf_stats {
    double *max_div, *max_div_in, *compat;
} ibf_stats;

typedef struct ibf_plan ibf_plan;

/* Build a plan for ngrids grids (1 <= ngrids <= IBF_MAX_GRIDS) on CUDA device `device`.
 * Validates every descriptor on the host, builds the z coefficients, the modified
 * wavenumbers, twiddle tables and the per-mode pivot tables of the tridiagonal
 * solves (float64 arithmetic), picks launch shapes (timed if opts->autotune),
 * and allocates all device workspace.  Synchronises the device.
 * On success *plan owns the workspace; on error *plan is NULL and nothing leaks.
 * Errors: INVALID_ARG, UNSUPPORTED_SIZE, UNSUPPORTED_BC, OOM, CUDA. */
ibf_status ibf_projection_plan(ibf_plan **plan, const ibf_grid *grids, int ngrids,
                               const ibf_opts *opts, int device);

/* Project grid g's u* = in[g] into out[g] (arrays of ngrids ibf_fields):
 * out.p <- phi (or the pressure update chosen by opts->pressure, reading p_n from
 * in[g].p; otherwise in[g].p is ignored), out.u/v/w <- u* - alpha dt G phi.  out may
 * alias in (in place).  dt > 0, alpha > 0.  stats may be NULL.  stream is a
 * cudaStream_t (NULL: legacy default stream).  Enqueues kernels only: no
 * allocation, no host synchronisation, so it can be captured into a CUDA graph.
 * Device-side errors are recorded in the plan and returned by
 * ibf_plan_sync_status.  Errors: INVALID_ARG, CUDA. */
ibf_status ibf_project(ibf_plan *plan, const ibf_fields *in, const ibf_fields *out,
                       double dt, double alpha, const ibf_stats *stats, void *stream);

/* Adjoint (vector-Jacobian product) of the map u* -> (u, phi) of ibf_project for the
 * Euclidean inner product:  grad_in = g_u + D^T S^-T (g_phi/(alpha dt) - G^T g_u),
 * S^-T = V S^-1 V^-1 with V = diag(dx dy hz_k), computed with the same solver.
 * grad_out[g].{u,v,w} = g_u (device, same shapes as the velocity), grad_out[g].p = g_phi
 * (may be NULL = zero).  The adjoint is that of the phi output: opts->pressure does not
 * enter it.  grad_in[g].{u,v,w} receive the gradient with respect to u*
 * (grad_in[g].p ignored).  grad_in may alias grad_out's velocity arrays.  Same
 * stream/capture rules as ibf_project. */
ibf_status ibf_project_backward(ibf_plan *plan, const ibf_fields *grad_out, const ibf_fields *grad_in,
                                double dt, double alpha, void *stream);

/* Factored implicit viscous solve (Section "Fluid Mechanics", Eq. nstime_discr with the
 * viscous terms advanced by Crank-Nicolson; Section "Fluid domain", provisional-step
 * paragraph: one tridiagonal solve per direction, Sherman-Morrison on the periodic
 * lines), for each velocity component c = u, v, w of every grid of the plan:
 *     out[g].c = (I - beta Lz)^-1 (I - beta Ly)^-1 (I - beta Lx)^-1 in[g].c,
 *     beta = alpha dt / (2 Re) >= 0,
 * with Lx, Ly the periodic second differences (spacing lx/nx, ly/ny; u on x-faces and
 * v on y-faces are periodic like the cells) and Lz the second difference of the
 * component's own z grid: for u and v the cell centres, no-slip walls at both z ends
 * (mirror ghost -f at distance hz from the first and last centre); for w the interior
 * faces 1..nz-1, whose wall faces 0 and nz are written as zero (in[g].w there is
 * ignored).  The x and y inverses are exact inverses of the periodic operators (taken
 * in the Fourier space of the projection's transforms); the z systems are solved by
 * Thomas' algorithm with pivots formed in fp64 on the device (again whenever beta
 * differs from the previous call's on this plan, and in every stream capture).
 * in / out: ngrids ibf_fields of DEVICE fp64 velocity arrays in the projection's
 * layouts (p and q ignored); out[g].c may alias in[g].c of the same component.
 * Precision: the plan's.  IBF_FP64 computes in fp64; IBF_MIXED runs the transforms
 * and the z sweeps in fp32 (fp64 input and output; relative error about 1e-6 of the
 * largest output value).  Uses the plan's workspace: same stream and capture rules as
 * ibf_project (no allocation, no host synchronisation).
 * Errors: INVALID_ARG (null plan or arrays, beta negative or not finite),
 * UNSUPPORTED_BC (a grid with a wall-bounded x or y), UNSUPPORTED_SIZE, CUDA. */
ibf_status ibf_viscous_solve(ibf_plan *plan, const ibf_fields *in, const ibf_fields *out, double beta,
                             void *stream);

/* Launch shape of one grid, chosen by ibf_projection_plan (defaults or, with
 * opts->autotune, the fastest candidate timed on this device), or forced by the
 * caller through ibf_projection_plan_tuned.  Every field <= 0 means "default".
 *   rows      : grid rows per CTA of the x-direction kernels (even);
 *   x_n1, y_n1: first factor of the two-level FFT along x / y (N = n1 * n2, both
 *               factors in {1,2,3,4,6,8,12,16,24,32});
 *   yz_kernel : 1 streaming y/z kernels (y-FFT fused with Thomas sweeps that stream
 *               the planes, the spectrum read and written twice), 2 resident slab
 *               (the whole z extent of a column block in shared memory: one read,
 *               one write; small grids only), 3 split (y-FFT of every (plane, column
 *               block) in its own CTA, then Thomas sweeps with one thread per mode:
 *               the spectrum read and written four times, all of it streamed),
 *               4 spectral z (uniform z with Neumann walls at both ends only, nz a
 *               product of two FFT sizes: the y-FFTs of 3, then per z line a DCT-II
 *               along z, division by the mode's eigenvalue, inverse DCT; no
 *               tridiagonal sweep; INVALID_ARG on a stretched z or an outlet);
 *   mb        : x-modes per column block of the y/z kernels;
 *   tri       : tridiagonal algorithm of the slab kernel: 1 Thomas per mode with the
 *               plan's pivot table, 1 + S (S >= 1) S levels of in-place cyclic
 *               reduction (all levels in parallel over modes and equations) before
 *               Thomas on the reduced systems; 1 + log2(nz) is full cyclic reduction. */
typedef struct ibf_tuning {
    int rows, x_n1, y_n1, yz_kernel, mb, tri;
} ibf_tuning;

/* ibf_projection_plan with the launch shape of every grid given (tuning: ngrids
 * entries, NULL = defaults; opts->autotune then only fills the fields left <= 0).
 * Errors as ibf_projection_plan; UNSUPPORTED_SIZE when a forced shape does not fit
 * the device (shared memory) or does not divide the grid. */
ibf_status ibf_projection_plan_tuned(ibf_plan **plan, const ibf_grid *grids, int ngrids,
                                     const ibf_opts *opts, int device, const ibf_tuning *tuning);

/* The launch shape grid g of the plan uses (all fields filled). */
ibf_status ibf_plan_get_tuning(const ibf_plan *plan, int g, ibf_tuning *out);

/* Synchronise the plan's last stream, return and clear the device error word
 * (IBF_OK, IBF_ERR_TIMEOUT, IBF_ERR_NONFINITE or IBF_WARN_INCOMPATIBLE_RHS). */
ibf_status ibf_plan_sync_status(ibf_plan *plan);

/* Release all workspace (synchronises the plan's device).  NULL is accepted. */
ibf_status ibf_plan_destroy(ibf_plan *plan);

/* Static description of a status code. */
const char *ibf_status_string(ibf_status s);

/* Text of the last CUDA error seen by this thread's calls (empty if none). */
const char *ibf_last_error(void);

/* Plan facts: workspace bytes, and per-grid launch choices. */
typedef struct ibf_plan_info {
    long long workspace_bytes;
    int ngrids;
    int precision;
    int refine_steps;
    long long total_cells;
} ibf_plan_info;
ibf_status ibf_plan_get_info(const ibf_plan *plan, ibf_plan_info *info);

/* Per-kernel timing with CUDA events recorded on the call's stream around every
 * launch (off by default).  ibf_profile_read fills up to `cap` entries: kernel
 * name (static string), launch count and summed milliseconds since the last
 * reset; it synchronises the plan's last stream.  Returns the number of entries. */
ibf_status ibf_profile_enable(ibf_plan *plan, int enable);
int ibf_profile_read(ibf_plan *plan, const char **names, long long *launches, double *ms, int cap);
ibf_status ibf_profile_reset(ibf_plan *plan);

/* ------------------------------------------------------------------------------
 * Projection without any device allocation (the paper has no counterpart; this is
 * a service of this library).
 *
 * For callers that may not allocate device memory when they project: a host
 * framework whose own allocator owns all of the GPU's memory, code running where an
 * allocation would synchronise the device or is not allowed, or loops that must not
 * pay for one.  ibf_projection_plan allocates its workspace; this entry point takes
 * the same workspace from one fixed device array of IBF_NOALLOC_SCRATCH_BYTES that
 * every GPU loading the library holds until the process exits.  It never calls
 * cudaMalloc/cudaFree or any allocating routine.
 *
 * Projects one grid like ibf_project (same layouts, conventions, precisions and
 * results; no statistics).  `in` and `out` are single ibf_fields of DEVICE pointers
 * (out may alias in); stream is a cudaStream_t or NULL.  The pivot table is rebuilt
 * on every call.  The call's small tables (grid descriptor, z metrics, twiddles) reach
 * the device as the arguments of copy-kernel launches on `stream`: no host memory is
 * read after the call returns, and the call does not wait for work already queued on
 * the stream.  Every call shares the one array and leaves its contents behind, so
 * calls that overlap on the GPU (other streams, other host threads) race and corrupt
 * each other: order them.  The first call on a device looks up the array's device
 * address and caches it; make that first call before any stream capture.
 * opts->pressure must be IBF_P_PHI.  Device-side conditions (a non-finite right-hand
 * side, an incompatible right-hand side) are not reported by this entry point: there
 * is no plan whose error word ibf_plan_sync_status could read.
 * Errors (all found on the host before anything is enqueued): INVALID_ARG,
 * UNSUPPORTED_BC, UNSUPPORTED_SIZE (also when the workspace of the grid does not fit
 * in IBF_NOALLOC_SCRATCH_BYTES: about 2.5 million cells in IBF_MIXED, 4.5 million in
 * IBF_FP64, or when a kernel's shared memory exceeds the limit ibf_projection_plan
 * applies); CUDA when a CUDA call fails. */
#define IBF_NOALLOC_SCRATCH_BYTES (64ull << 20)
ibf_status ibf_project_noalloc(const ibf_grid *grid, const ibf_opts *opts, const ibf_fields *in,
                               const ibf_fields *out, double dt, double alpha, void *stream);

#ifdef __cplusplus
}
#endif
#endif /* IBF_H */

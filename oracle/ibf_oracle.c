/*
 * ibf_oracle.c -- plain FP64 CPU oracle for the staggered-grid pressure projection.
 *
 * TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and the CPU
 * baseline leg of bench.py load this library.  The product (the CUDA library in
 * paper_2609_19130_gb300/csrc) never includes, links or calls anything here, and
 * this file includes nothing from it.
 *
 * What it computes (IB-Flows, Section "Fluid Mechanics"):
 *   Eq. (elliptic):  lap(phi) = (div u* - q) / (alpha dt),  q = 0
 *   Eq. (velsolen):  u_{n+1} = u* - alpha dt grad(phi)
 * on the staggered Cartesian grid with 2nd-order centred differences, x1,x2
 * periodic and uniform, x3 bounded by walls with a non-uniform spacing and a
 * homogeneous Neumann condition for phi; "the arbitrary constant of phi is
 * removed by fixing a reference value" (same section, boundary-condition
 * paragraph).  The Poisson equation is solved the way the paper describes its
 * solver (Section "Fluid domain", projection paragraph): Fourier transforms in
 * the two periodic directions leave one tridiagonal system along x3 per
 * horizontal mode.  Here the transforms are NAIVE O(N^2) DFT sums (and a naive
 * DCT-II/III for the optional wall-bounded x or y direction) and each
 * tridiagonal system is solved with the textbook Thomas algorithm, in FP64,
 * one real system for the real part and one for the imaginary part.
 *
 * Readings taken where the paper is silent:
 *  R1 index convention: cells i<nx, j<ny, k<nz; u[k][j][i] sits on the x-face
 *     at x = i dx (face i is the left face of cell i), v on the y-face at
 *     y = j dy, w[k][j][i] on the z-face z = zf[k], k = 0..nz (w[0], w[nz] are
 *     the walls); phi, b at cell centres; zc_k = (zf_k + zf_{k+1}) / 2.
 *  R2 operators: (D u)_c = (u_{i+1}-u_i)/dx + (v_{j+1}-v_j)/dy + (w_{k+1}-w_k)/hz_k;
 *     (G phi) on interior faces = difference of the two adjacent cells divided
 *     by dx, dy or gz_k = zc_k - zc_{k-1}; G is 0 on wall faces (Neumann), so
 *     the projection leaves the imposed wall-normal velocity unchanged.
 *     L = D G.
 *  R3 reference value: the volume-weighted mean of b is removed first
 *     (compatibility; its value is reported), the (0,0) mode is solved with
 *     its first level pinned to zero, and the volume-weighted mean of phi is
 *     removed at the end, so sum_c V_c phi_c = 0 with V_c = dx dy hz_k.
 *  R4 wall-bounded x (or y), not used by the paper: u has nx+1 faces,
 *     u[..][..][0] and u[..][..][nx] are walls, and the x transform is DCT-II.
 *  R5 tanh stretching: zf_k = lz/2 (1 + tanh(beta (2k/nz - 1)) / tanh(beta)).
 *  R6 Dirichlet outlet (boundary-condition paragraph of the same section: with
 *     neumann_velocity the pressure-correction equation takes a homogeneous
 *     Dirichlet condition at the outlet): phi = 0 on the top face z = lz, taken
 *     through the mirror value -phi_{nz-1}, so G phi on the top face is
 *     -phi_{nz-1} / (lz - zc_{nz-1}) and the top face velocity is corrected.  L is
 *     then nonsingular: no compatibility mean is removed and no reference value is
 *     fixed.
 *
 * Build: gcc -O2 -fopenmp -ffp-contract=off -shared -fPIC (see build_oracle.py).
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

#define IBFO_PI 3.14159265358979323846

typedef struct {
    int nx, ny, nz;
    double lx, ly;
    const double *zf;   /* nz+1 ascending face coordinates */
    int wall_x, wall_y; /* 0: periodic, 1: walls (Neumann phi, DCT) */
    int dirichlet_top;  /* 0: Neumann phi at z = lz; 1: phi = 0 there (R6) */
} ibfo_grid;

/* ------------------------------------------------------------------ grid */

void ibfo_zfaces_tanh(int nz, double lz, double beta, double *zf)
{
    for (int k = 0; k <= nz; ++k) {
        if (beta == 0.0)
            zf[k] = lz * (double)k / (double)nz;
        else
            zf[k] = 0.5 * lz * (1.0 + tanh(beta * (2.0 * k / nz - 1.0)) / tanh(beta));
    }
    zf[0] = 0.0;
    zf[nz] = lz;
}

static int nxu_of(const ibfo_grid *g) { return g->wall_x ? g->nx + 1 : g->nx; }
static int nyv_of(const ibfo_grid *g) { return g->wall_y ? g->ny + 1 : g->ny; }

static double hz_of(const ibfo_grid *g, int k) { return g->zf[k + 1] - g->zf[k]; }
static double zc_of(const ibfo_grid *g, int k) { return 0.5 * (g->zf[k] + g->zf[k + 1]); }
static double gz_of(const ibfo_grid *g, int k) { return zc_of(g, k) - zc_of(g, k - 1); } /* 1<=k<=nz-1 */
/* distance from the last cell centre to the top face (R6) */
static double gtop_of(const ibfo_grid *g) { return g->zf[g->nz] - zc_of(g, g->nz - 1); }

/* ------------------------------------------------------- R2: D, G, L */

/* div[k][j][i] = (D u)_c */
void ibfo_divergence(const ibfo_grid *g, const double *u, const double *v, const double *w, double *div)
{
    const int nx = g->nx, ny = g->ny, nz = g->nz, nxu = nxu_of(g), nyv = nyv_of(g);
    const double dx = g->lx / nx, dy = g->ly / ny;
    #pragma omp parallel for schedule(static)
    for (int k = 0; k < nz; ++k) {
        const double hz = hz_of(g, k);
        for (int j = 0; j < ny; ++j)
            for (int i = 0; i < nx; ++i) {
                int ip = g->wall_x ? i + 1 : (i + 1) % nx;
                int jp = g->wall_y ? j + 1 : (j + 1) % ny;
                double du = u[((size_t)k * ny + j) * nxu + ip] - u[((size_t)k * ny + j) * nxu + i];
                double dv = v[((size_t)k * nyv + jp) * nx + i] - v[((size_t)k * nyv + j) * nx + i];
                double dw = w[((size_t)(k + 1) * ny + j) * nx + i] - w[((size_t)k * ny + j) * nx + i];
                div[((size_t)k * ny + j) * nx + i] = du / dx + dv / dy + dw / hz;
            }
    }
}

/* (gu, gv, gw) = G phi; wall faces get 0. */
void ibfo_gradient(const ibfo_grid *g, const double *phi, double *gu, double *gv, double *gw)
{
    const int nx = g->nx, ny = g->ny, nz = g->nz, nxu = nxu_of(g), nyv = nyv_of(g);
    const double dx = g->lx / nx, dy = g->ly / ny;
    #pragma omp parallel for schedule(static)
    for (int k = 0; k < nz; ++k) {
        for (int j = 0; j < ny; ++j)
            for (int i = 0; i < nxu; ++i) {
                double val;
                if (g->wall_x && (i == 0 || i == nx)) val = 0.0;
                else {
                    int im = (i - 1 + nx) % nx;
                    val = (phi[((size_t)k * ny + j) * nx + (i % nx)] - phi[((size_t)k * ny + j) * nx + im]) / dx;
                }
                gu[((size_t)k * ny + j) * nxu + i] = val;
            }
        for (int j = 0; j < nyv; ++j)
            for (int i = 0; i < nx; ++i) {
                double val;
                if (g->wall_y && (j == 0 || j == ny)) val = 0.0;
                else {
                    int jm = (j - 1 + ny) % ny;
                    val = (phi[((size_t)k * ny + (j % ny)) * nx + i] - phi[((size_t)k * ny + jm) * nx + i]) / dy;
                }
                gv[((size_t)k * nyv + j) * nx + i] = val;
            }
    }
    #pragma omp parallel for schedule(static)
    for (int k = 0; k <= nz; ++k) {
        for (int j = 0; j < ny; ++j)
            for (int i = 0; i < nx; ++i) {
                double val = 0.0;
                if (k > 0 && k < nz)
                    val = (phi[((size_t)k * ny + j) * nx + i] - phi[((size_t)(k - 1) * ny + j) * nx + i]) / gz_of(g, k);
                else if (k == nz && g->dirichlet_top)
                    val = (0.0 - phi[((size_t)(k - 1) * ny + j) * nx + i]) / gtop_of(g);
                gw[((size_t)k * ny + j) * nx + i] = val;
            }
    }
}

static size_t ncell(const ibfo_grid *g) { return (size_t)g->nx * g->ny * g->nz; }
static size_t nu_of(const ibfo_grid *g) { return (size_t)g->nz * g->ny * nxu_of(g); }
static size_t nv_of(const ibfo_grid *g) { return (size_t)g->nz * nyv_of(g) * g->nx; }
static size_t nw_of(const ibfo_grid *g) { return (size_t)(g->nz + 1) * g->ny * g->nx; }

/* out = L phi = D (G phi) */
void ibfo_laplacian(const ibfo_grid *g, const double *phi, double *out)
{
    double *gu = malloc(nu_of(g) * sizeof(double));
    double *gv = malloc(nv_of(g) * sizeof(double));
    double *gw = malloc(nw_of(g) * sizeof(double));
    ibfo_gradient(g, phi, gu, gv, gw);
    ibfo_divergence(g, gu, gv, gw, out);
    free(gu); free(gv); free(gw);
}

/* Transposes of G and D, written as scatters over the same stencils (used by
 * the adjoint projection). */
void ibfo_gradient_T(const ibfo_grid *g, const double *gu, const double *gv, const double *gw, double *out)
{
    const int nx = g->nx, ny = g->ny, nz = g->nz, nxu = nxu_of(g), nyv = nyv_of(g);
    const double dx = g->lx / nx, dy = g->ly / ny;
    memset(out, 0, ncell(g) * sizeof(double));
    for (int k = 0; k < nz; ++k)
        for (int j = 0; j < ny; ++j) {
            for (int i = 0; i < nxu; ++i) {
                if (g->wall_x && (i == 0 || i == nx)) continue;
                double f = gu[((size_t)k * ny + j) * nxu + i] / dx;
                int ic = i % nx, im = (i - 1 + nx) % nx;
                out[((size_t)k * ny + j) * nx + ic] += f;
                out[((size_t)k * ny + j) * nx + im] -= f;
            }
        }
    for (int k = 0; k < nz; ++k)
        for (int j = 0; j < nyv; ++j) {
            if (g->wall_y && (j == 0 || j == ny)) continue;
            int jc = j % ny, jm = (j - 1 + ny) % ny;
            for (int i = 0; i < nx; ++i) {
                double f = gv[((size_t)k * nyv + j) * nx + i] / dy;
                out[((size_t)k * ny + jc) * nx + i] += f;
                out[((size_t)k * ny + jm) * nx + i] -= f;
            }
        }
    for (int k = 1; k < nz; ++k) {
        double rg = 1.0 / gz_of(g, k);
        for (int j = 0; j < ny; ++j)
            for (int i = 0; i < nx; ++i) {
                double f = gw[((size_t)k * ny + j) * nx + i] * rg;
                out[((size_t)k * ny + j) * nx + i] += f;
                out[((size_t)(k - 1) * ny + j) * nx + i] -= f;
            }
    }
    if (g->dirichlet_top) {
        double rg = 1.0 / gtop_of(g);
        for (int j = 0; j < ny; ++j)
            for (int i = 0; i < nx; ++i)
                out[((size_t)(nz - 1) * ny + j) * nx + i] -= gw[((size_t)nz * ny + j) * nx + i] * rg;
    }
}

void ibfo_divergence_T(const ibfo_grid *g, const double *c, double *gu, double *gv, double *gw)
{
    const int nx = g->nx, ny = g->ny, nz = g->nz, nxu = nxu_of(g), nyv = nyv_of(g);
    const double dx = g->lx / nx, dy = g->ly / ny;
    memset(gu, 0, nu_of(g) * sizeof(double));
    memset(gv, 0, nv_of(g) * sizeof(double));
    memset(gw, 0, nw_of(g) * sizeof(double));
    for (int k = 0; k < nz; ++k) {
        double hz = hz_of(g, k);
        for (int j = 0; j < ny; ++j)
            for (int i = 0; i < nx; ++i) {
                double s = c[((size_t)k * ny + j) * nx + i];
                int ip = g->wall_x ? i + 1 : (i + 1) % nx;
                int jp = g->wall_y ? j + 1 : (j + 1) % ny;
                gu[((size_t)k * ny + j) * nxu + ip] += s / dx;
                gu[((size_t)k * ny + j) * nxu + i] -= s / dx;
                gv[((size_t)k * nyv + jp) * nx + i] += s / dy;
                gv[((size_t)k * nyv + j) * nx + i] -= s / dy;
                gw[((size_t)(k + 1) * ny + j) * nx + i] += s / hz;
                gw[((size_t)k * ny + j) * nx + i] -= s / hz;
            }
    }
}

/* ------------------------------------------------- naive 1-D transforms */

typedef struct { double re, im; } cplx;

/* Forward DFT  F_m = sum_n f_n exp(-2 pi i m n / N); inverse adds +, scales 1/N.
 * Twiddles from a table of exp(-2 pi i r / N), index (m n) mod N. */
static void dft_naive(const cplx *in, cplx *out, int n, int inverse, const cplx *tw)
{
    for (int m = 0; m < n; ++m) {
        double sr = 0.0, si = 0.0;
        for (int t = 0; t < n; ++t) {
            cplx w = tw[(int)(((long long)m * t) % n)];
            double wi = inverse ? -w.im : w.im;
            sr += in[t].re * w.re - in[t].im * wi;
            si += in[t].re * wi + in[t].im * w.re;
        }
        if (inverse) { sr /= n; si /= n; }
        out[m].re = sr; out[m].im = si;
    }
}

/* DCT-II  F_m = sum_n f_n cos(pi m (2n+1) / (2N)),
 * inverse (DCT-III)  f_n = (1/N) [F_0 + 2 sum_{m>=1} F_m cos(pi m (2n+1) / (2N))].
 * Table cs[r] = cos(pi r / (2N)), index (m (2n+1)) mod 4N.  Applied to the real
 * and imaginary parts independently. */
static void dct_naive(const cplx *in, cplx *out, int n, int inverse, const double *cs)
{
    for (int a = 0; a < n; ++a) {
        double sr = 0.0, si = 0.0;
        if (!inverse) {
            for (int t = 0; t < n; ++t) {
                double c = cs[(int)(((long long)a * (2 * t + 1)) % (4 * n))];
                sr += in[t].re * c; si += in[t].im * c;
            }
        } else {
            for (int m = 0; m < n; ++m) {
                double c = cs[(int)(((long long)m * (2 * a + 1)) % (4 * n))];
                double wgt = (m == 0) ? 1.0 : 2.0;
                sr += wgt * in[m].re * c; si += wgt * in[m].im * c;
            }
            sr /= n; si /= n;
        }
        out[a].re = sr; out[a].im = si;
    }
}

typedef struct {
    int n, is_dct;
    cplx *tw;    /* n entries (DFT) */
    double *cs;  /* 4n entries (DCT) */
} xform;

static void xform_init(xform *x, int n, int is_dct)
{
    x->n = n; x->is_dct = is_dct; x->tw = NULL; x->cs = NULL;
    if (is_dct) {
        x->cs = malloc(sizeof(double) * 4 * n);
        for (int r = 0; r < 4 * n; ++r) x->cs[r] = cos(IBFO_PI * r / (2.0 * n));
    } else {
        x->tw = malloc(sizeof(cplx) * n);
        for (int r = 0; r < n; ++r) { x->tw[r].re = cos(2.0 * IBFO_PI * r / n); x->tw[r].im = -sin(2.0 * IBFO_PI * r / n); }
    }
}
static void xform_free(xform *x) { free(x->tw); free(x->cs); }
static void xform_apply(const xform *x, const cplx *in, cplx *out, int inverse)
{
    if (x->is_dct) dct_naive(in, out, x->n, inverse, x->cs);
    else dft_naive(in, out, x->n, inverse, x->tw);
}

/* exported for the transform pins: one naive transform of length n */
void ibfo_dft(const double *in_re, const double *in_im, double *out_re, double *out_im, int n, int inverse, int is_dct)
{
    xform x; xform_init(&x, n, is_dct);
    cplx *a = malloc(sizeof(cplx) * n), *b = malloc(sizeof(cplx) * n);
    for (int t = 0; t < n; ++t) { a[t].re = in_re[t]; a[t].im = in_im ? in_im[t] : 0.0; }
    xform_apply(&x, a, b, inverse);
    for (int t = 0; t < n; ++t) { out_re[t] = b[t].re; out_im[t] = b[t].im; }
    free(a); free(b); xform_free(&x);
}

/* eigenvalue of the 1-D second difference for mode m (DFT or DCT basis) */
static double lambda_1d(int m, int n, double h, int is_dct)
{
    double s = is_dct ? sin(IBFO_PI * m / (2.0 * n)) : sin(IBFO_PI * m / n);
    return -4.0 / (h * h) * s * s;
}

/* ------------------------------------------------------------ Thomas */

/* Solve a_k x_{k-1} + d_k x_k + c_k x_{k+1} = r_k for k = k0..n-1, with
 * x_{k0-1} treated as 0 (a_{k0} ignored).  Textbook forward elimination and
 * back substitution.  x[0..k0-1] are set to 0. */
static void thomas(const double *a, const double *d, const double *c, const double *r, double *x,
                   int n, int k0, double *cp, double *dp)
{
    for (int k = 0; k < k0; ++k) x[k] = 0.0;
    if (k0 >= n) return;
    cp[k0] = c[k0] / d[k0];
    dp[k0] = r[k0] / d[k0];
    for (int k = k0 + 1; k < n; ++k) {
        double den = d[k] - a[k] * cp[k - 1];
        cp[k] = c[k] / den;
        dp[k] = (r[k] - a[k] * dp[k - 1]) / den;
    }
    x[n - 1] = dp[n - 1];
    for (int k = n - 2; k >= k0; --k) x[k] = dp[k] - cp[k] * x[k + 1];
}

/* ------------------------------------------------------- Poisson solve */

/* phi = S^-1 b : the unique phi with L phi = b - <b>_V and <phi>_V = 0
 * (reading R3), or with a Dirichlet outlet (R6) the unique phi with L phi = b.
 * Returns the removed <b>_V (0 with a Dirichlet outlet) in *compat.  b is not
 * modified. */
int ibfo_poisson(const ibfo_grid *g, const double *b, double *phi, double *compat)
{
    const int nx = g->nx, ny = g->ny, nz = g->nz;
    const double dx = g->lx / nx, dy = g->ly / ny;
    const size_t plane = (size_t)nx * ny;

    /* z coefficients of L along x3: a_k phi_{k-1} + (-(a_k+c_k)) phi_k + c_k phi_{k+1} */
    double *az = calloc(nz, sizeof(double)), *cz = calloc(nz, sizeof(double)), *bz = calloc(nz, sizeof(double));
    double sumV = 0.0, sumVb = 0.0;
    for (int k = 0; k < nz; ++k) {
        double hz = hz_of(g, k);
        az[k] = (k > 0) ? 1.0 / (hz * gz_of(g, k)) : 0.0;
        cz[k] = (k < nz - 1) ? 1.0 / (hz * gz_of(g, k + 1)) : 0.0;
        bz[k] = -(az[k] + cz[k]);
        if (k == nz - 1 && g->dirichlet_top) bz[k] -= 1.0 / (hz * gtop_of(g));  /* flux to phi = 0 */
        double s = 0.0;
        for (size_t p = 0; p < plane; ++p) s += b[(size_t)k * plane + p];
        sumVb += hz * s;          /* dx dy cancels in the weighted mean */
        sumV += hz * (double)plane;
    }
    const double mean_b = g->dirichlet_top ? 0.0 : sumVb / sumV;
    if (compat) *compat = mean_b;

    /* spectral coefficients: spec[k][n][m] */
    cplx *spec = malloc(sizeof(cplx) * plane * nz);
    xform tx, ty;
    xform_init(&tx, nx, g->wall_x);
    xform_init(&ty, ny, g->wall_y);

    /* forward: x along rows, then y along columns, plane by plane */
    #pragma omp parallel
    {
        cplx *rin = malloc(sizeof(cplx) * (nx > ny ? nx : ny));
        cplx *rout = malloc(sizeof(cplx) * (nx > ny ? nx : ny));
        #pragma omp for schedule(static)
        for (int k = 0; k < nz; ++k) {
            cplx *P = spec + (size_t)k * plane;
            for (int j = 0; j < ny; ++j) {
                for (int i = 0; i < nx; ++i) { rin[i].re = b[(size_t)k * plane + (size_t)j * nx + i] - mean_b; rin[i].im = 0.0; }
                xform_apply(&tx, rin, rout, 0);
                for (int m = 0; m < nx; ++m) P[(size_t)j * nx + m] = rout[m];
            }
            for (int m = 0; m < nx; ++m) {
                for (int j = 0; j < ny; ++j) rin[j] = P[(size_t)j * nx + m];
                xform_apply(&ty, rin, rout, 0);
                for (int n = 0; n < ny; ++n) P[(size_t)n * nx + m] = rout[n];
            }
        }
        free(rin); free(rout);
    }

    /* one tridiagonal system along x3 per horizontal mode (m, n) */
    #pragma omp parallel
    {
        double *d = malloc(sizeof(double) * nz), *r = malloc(sizeof(double) * nz), *x = malloc(sizeof(double) * nz);
        double *cp = malloc(sizeof(double) * nz), *dp = malloc(sizeof(double) * nz);
        #pragma omp for schedule(static)
        for (long long mode = 0; mode < (long long)plane; ++mode) {
            int n = (int)(mode / nx), m = (int)(mode % nx);
            double lam = lambda_1d(m, nx, dx, g->wall_x) + lambda_1d(n, ny, dy, g->wall_y);
            int k0 = (m == 0 && n == 0 && !g->dirichlet_top) ? 1 : 0;   /* pin the first level of the singular mode */
            for (int k = 0; k < nz; ++k) d[k] = bz[k] + lam;
            for (int part = 0; part < 2; ++part) {
                for (int k = 0; k < nz; ++k) {
                    cplx z = spec[(size_t)k * plane + mode];
                    r[k] = part ? z.im : z.re;
                }
                thomas(az, d, cz, r, x, nz, k0, cp, dp);
                for (int k = 0; k < nz; ++k) {
                    if (part) spec[(size_t)k * plane + mode].im = x[k];
                    else spec[(size_t)k * plane + mode].re = x[k];
                }
            }
        }
        free(d); free(r); free(x); free(cp); free(dp);
    }

    /* inverse: y then x */
    #pragma omp parallel
    {
        cplx *rin = malloc(sizeof(cplx) * (nx > ny ? nx : ny));
        cplx *rout = malloc(sizeof(cplx) * (nx > ny ? nx : ny));
        #pragma omp for schedule(static)
        for (int k = 0; k < nz; ++k) {
            cplx *P = spec + (size_t)k * plane;
            for (int m = 0; m < nx; ++m) {
                for (int n = 0; n < ny; ++n) rin[n] = P[(size_t)n * nx + m];
                xform_apply(&ty, rin, rout, 1);
                for (int j = 0; j < ny; ++j) P[(size_t)j * nx + m] = rout[j];
            }
            for (int j = 0; j < ny; ++j) {
                for (int m = 0; m < nx; ++m) rin[m] = P[(size_t)j * nx + m];
                xform_apply(&tx, rin, rout, 1);
                for (int i = 0; i < nx; ++i) phi[(size_t)k * plane + (size_t)j * nx + i] = rout[i].re;
            }
        }
        free(rin); free(rout);
    }

    /* remove the volume-weighted mean of phi */
    double sVp = 0.0;
    for (int k = 0; k < nz; ++k) {
        double s = 0.0;
        for (size_t p = 0; p < plane; ++p) s += phi[(size_t)k * plane + p];
        sVp += hz_of(g, k) * s;
    }
    const double mean_phi = g->dirichlet_top ? 0.0 : sVp / sumV;
    for (size_t c = 0; c < plane * nz; ++c) phi[c] -= mean_phi;

    xform_free(&tx); xform_free(&ty);
    free(spec); free(az); free(bz); free(cz);
    return 0;
}

/* ---------------------------------------------------------- projection */

static double maxabs(const double *a, size_t n)
{
    double m = 0.0;
    for (size_t t = 0; t < n; ++t) { double v = fabs(a[t]); if (v > m || v != v) m = v; }
    return m;
}

/* stats (nullable, 4 doubles): [0] max|D u| after, [1] max|D u*|, [2] <b>_V removed, [3] 0 */
int ibfo_project(const ibfo_grid *g, const double *us, const double *vs, const double *ws,
                 double dt, double alpha, double *phi, double *u, double *v, double *w, double *stats)
{
    const size_t nc = ncell(g), nu = nu_of(g), nv = nv_of(g), nw = nw_of(g);
    const double s = alpha * dt;
    double *b = malloc(nc * sizeof(double));
    ibfo_divergence(g, us, vs, ws, b);
    double maxdiv_in = maxabs(b, nc);
    for (size_t c = 0; c < nc; ++c) b[c] /= s;          /* Eq. (elliptic), q = 0 */
    double compat = 0.0;
    ibfo_poisson(g, b, phi, &compat);
    double *gu = malloc(nu * sizeof(double)), *gv = malloc(nv * sizeof(double)), *gw = malloc(nw * sizeof(double));
    ibfo_gradient(g, phi, gu, gv, gw);
    for (size_t t = 0; t < nu; ++t) u[t] = us[t] - s * gu[t];   /* Eq. (velsolen) */
    for (size_t t = 0; t < nv; ++t) v[t] = vs[t] - s * gv[t];
    for (size_t t = 0; t < nw; ++t) w[t] = ws[t] - s * gw[t];
    if (stats) {
        ibfo_divergence(g, u, v, w, b);
        stats[0] = maxabs(b, nc);
        stats[1] = maxdiv_in;
        stats[2] = compat;
        stats[3] = 0.0;
    }
    free(b); free(gu); free(gv); free(gw);
    return 0;
}

/* Adjoint of the projection u* -> (u, phi) for the Euclidean inner product:
 *   gbar = g_u + D^T S^-T (g_phi/(alpha dt) - G^T g_u),   S^-T = V S^-1 V^-1,
 * with V = diag(dx dy hz_k) (L is V-self-adjoint because D = -V^-1 G^T V_f,
 * and both weighted-mean removals are V-orthogonal projectors).
 * g_phi may be NULL (treated as zero). */
int ibfo_project_adjoint(const ibfo_grid *g, const double *gu, const double *gv, const double *gw,
                         const double *gphi, double dt, double alpha,
                         double *gus, double *gvs, double *gws)
{
    const size_t nc = ncell(g), nu = nu_of(g), nv = nv_of(g), nw = nw_of(g);
    const size_t plane = (size_t)g->nx * g->ny;
    const double s = alpha * dt;
    double *h = malloc(nc * sizeof(double)), *psi = malloc(nc * sizeof(double));
    ibfo_gradient_T(g, gu, gv, gw, h);
    for (size_t c = 0; c < nc; ++c) h[c] = (gphi ? gphi[c] / s : 0.0) - h[c];
    for (int k = 0; k < g->nz; ++k) {                 /* V^-1 (dx dy cancels) */
        double r = 1.0 / hz_of(g, k);
        for (size_t p = 0; p < plane; ++p) h[(size_t)k * plane + p] *= r;
    }
    ibfo_poisson(g, h, psi, NULL);
    for (int k = 0; k < g->nz; ++k) {                 /* V */
        double hz = hz_of(g, k);
        for (size_t p = 0; p < plane; ++p) psi[(size_t)k * plane + p] *= hz;
    }
    ibfo_divergence_T(g, psi, gus, gvs, gws);
    for (size_t t = 0; t < nu; ++t) gus[t] += gu[t];
    for (size_t t = 0; t < nv; ++t) gvs[t] += gv[t];
    for (size_t t = 0; t < nw; ++t) gws[t] += gw[t];
    free(h); free(psi);
    return 0;
}

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
#include "ibf_common.cuh"

#include <type_traits>

namespace ibf {

// ================================================================ k_xfwd
constexpr int kRowGroup = 4;  // rows whose loads are issued together (memory-level parallelism)

// Right-hand side of one solve for a block of rows of plane k, then the real FFT
// along x of the rows (two rows per complex transform), stored as x-modes.
// W: the launch contains wall-bounded grids (compiled out of periodic-only plans).
// SPLIT = 2 (mixed path, rows divisible by 4): two CTAs of kXThreads / 2 threads per
// row block, each forming and transforming half of its rows, so that one CTA's
// transform overlaps another's loads; each half writes its own plane-sum slot.  Five
// half-block CTAs per SM (96 registers: 20 warps to hide latency) except for the later
// sweeps' residuals, whose stencils need the 128 registers of four.
template <typename T, class A, int MODE, bool W, int SPLIT>
__global__ void __launch_bounds__(kXThreads / SPLIT, SPLIT == 2 ? ((MODE == XM_RESID || MODE == XM_RESID1) ? 4 : 5)
                                                               : (sizeof(T) == 4 ? 2 : 1))
    k_xfwd(Work w, UserPtrs p, int use_ws, int lo_valid, double s, double rs) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    cx<T> *buf = reinterpret_cast<cx<T> *>(smem_raw);
    __shared__ double red[kXThreads / 32];
    __shared__ float redf[kXThreads / 32];
    typedef typename A::V V;

    const int b = blockIdx.x / SPLIT + p.blk0;
    const int half = SPLIT == 2 ? (int)(blockIdx.x & 1u) : 0;
    const int g = find_grid(w.xblk_start, w.ngrids, b);
    const GridDev &G = w.grids[g];
    const int lb = b - __ldg(w.xblk_start + g);
    const int nrb = G.nrb, rows = G.rows / SPLIT;
    const int k = lb / nrb, rb = lb - k * nrb;
    const int j0 = rb * G.rows + half * rows;
    const int nx = G.nx, ny = G.ny, nz = G.nz;
    // sequences one complex element further apart than their length, so that the
    // split / gather steps, which read the same position of several sequences, do not
    // fall into one shared-memory bank
    const int N1 = G.nx1, N2 = G.nx2, sstride = fft_seq_len(N1, N2) + 1;
    const FDiv fN1 = G.fnx1, fN2 = G.fnx2;
    const int gi = g - p.g0;
    const int zo = G.z_off;
    const ptrdiff_t plane = (ptrdiff_t)nx * ny;
    const ptrdiff_t pbase = (ptrdiff_t)k * plane;
    const int wall_x = W ? G.wall_x : 0, wall_y = W ? G.wall_y : 0, nxu = W ? G.nxu : nx;

    // the first right-hand side (Eq. elliptic): (D u* - q)/(alpha dt), q = 0 in XM_DIV
    constexpr bool DIVL = MODE == XM_DIV || MODE == XM_DIVQ;
    V cu, cv, cwp, cwm, cp;
    if (DIVL) {
        const double rhz = w.z.rhz[zo + k];
        cu = Coef<A>::c(rs * G.rdx);
        cv = Coef<A>::c(rs * G.rdy);
        cwp = Coef<A>::c(rs * rhz);
        cwm = cwp;
        cp = Coef<A>::c(-rs);
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
        // right neighbour: the next face of the u row (face nx when x is wall-bounded) on
        // the divergence paths, the next cell (periodic wrap) on the residual path
        const int ip = (ii + 1 == nx && (MODE == XM_RESID || MODE == XM_RESID0 || MODE == XM_RESID1 || !wall_x)) ? 0 : ii + 1;
        const int im = (ii == 0) ? nx - 1 : ii - 1;
        const bool own_up = (lane == 31) || (ii + 1 == nx);
        const bool own_dn = (lane == 0) || (ii == 0);
        const int spos = pos_nat(wall_x ? dct_perm(ii, nx) : ii, fN2);
        if constexpr (MODE == XM_COPY) {
            // the field itself, one row after the other (plane k + zshift; zero past the
            // last interior face of w)
            const bool live = !(p.zshift && k == nz - 1);
            const double *src = p.in_u[gi] + (ptrdiff_t)(k + p.zshift) * plane;
            for (int jg = sm.r0; jg < sm.r1; jg += kRowGroup) {
                double v[kRowGroup];
#pragma unroll
                for (int q = 0; q < kRowGroup; ++q) {
                    const int jl = jg + q, j = j0 + jl;
                    v[q] = (act && live && jl < sm.r1 && j < ny) ? __ldg(src + (ptrdiff_t)j * nx + i) : 0.0;
                }
#pragma unroll
                for (int q = 0; q < kRowGroup; ++q) {
                    const int jl = jg + q;
                    if (jl >= sm.r1) break;
                    if (act) *(reinterpret_cast<T *>(buf + (jl >> 1) * sstride + spos) + (jl & 1)) = (T)v[q] * scale;
                }
            }
        } else if (DIVL || MODE == XM_ADJ) {
            // wall-bounded x: u rows hold nx+1 faces; wall-bounded y: v planes hold ny+1 rows
            const double *u = p.in_u[gi] + (ptrdiff_t)k * ny * nxu;
            const double *vv = p.in_v[gi] + (ptrdiff_t)k * (W ? G.nyv : ny) * nx, *ww = p.in_w[gi] + pbase;
            // adjoint source: G^T skips wall faces (G is zero there)
            const bool zero_u = MODE == XM_ADJ && wall_x && ii == 0;
            const bool zero_un = MODE == XM_ADJ && wall_x && ii + 1 == nx;
            // extra cell-centred source: g_phi (adjoint) or the mass source q
            const double *psrc = MODE == XM_ADJ ? p.in_p[gi] : (MODE == XM_DIVQ ? p.in_q[gi] : nullptr);
            const double *pp = psrc ? psrc + pbase : nullptr;
            V vcur = A::zero();
            double vcur64 = 0.0;  // float-float divergence: v of the current row, fp64
            bool have_v = false;
            df2 acc2 = {make_float2(0.f, 0.f), make_float2(0.f, 0.f)};  // float-float divergence: plane sum, per lane
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
                        const int jp = (j + 1 == ny && !wall_y) ? 0 : j + 1;
                        const int row = j * nx, rowu = j * nxu;
                        ru[q] = __ldg(u + rowu + ii);
                        if (own_up) rue[q] = __ldg(u + rowu + ip);
                        if (q == 0 && need_v0) rv0 = __ldg(vv + row + ii);
                        rvn[q] = __ldg(vv + jp * nx + ii);
                        rw0[q] = __ldg(ww + row + ii);
                        rw1[q] = __ldg(ww + plane + row + ii);
                        if ((MODE == XM_ADJ || MODE == XM_DIVQ) && pp) rp[q] = __ldg(pp + row + ii);
                    }
                }
                if (need_v0) {
                    if constexpr (IsDF<A>::value && DIVL) vcur64 = rv0;
                    else vcur = A::load(rv0);
                }
                if constexpr (IsDF<A>::value && DIVL) {
                // float-float divergence, two rows at a time: the three face differences of
                // each row in fp64 (three DADD per cell, each rounded to 2^-53 of the
                // difference), the coefficient products per row, every sum of both rows in
                // two-lane operations (bit for bit the scalar sequence)
#pragma unroll
                for (int q = 0; q < kRowGroup; q += 2) {
                    const int jl0 = jg + q;
                    if (jl0 >= sm.r1) break;  // warp-uniform
                    df d1[2], d2[2], d3[2], dq[2];
                    bool live[2];
#pragma unroll
                    for (int h = 0; h < 2; ++h) {
                        const int j = j0 + jl0 + h;
                        live[h] = jl0 + h < sm.r1 && j < ny;
                        double Un = __shfl_down_sync(0xffffffffu, ru[q + h], 1);
                        if (own_up) Un = rue[q + h];
                        const double Vc = vcur64;
                        d1[h] = f64_to_df(__dsub_rn(Un, ru[q + h]));
                        d2[h] = f64_to_df(__dsub_rn(rvn[q + h], Vc));
                        d3[h] = f64_to_df(__dsub_rn(rw1[q + h], rw0[q + h]));
                        if (MODE == XM_DIVQ && pp) dq[h] = A::mul(cp, A::load(rp[q + h]));
                        if (live[h]) {
                            vcur64 = rvn[q + h];
                            have_v = true;
                        } else {
                            have_v = false;
                        }
                    }
                    df2 bv = df_dot3_2(cu, df2{make_float2(d1[0].hi, d1[1].hi), make_float2(d1[0].lo, d1[1].lo)},
                                       cv, df2{make_float2(d2[0].hi, d2[1].hi), make_float2(d2[0].lo, d2[1].lo)},
                                       cwp, df2{make_float2(d3[0].hi, d3[1].hi), make_float2(d3[0].lo, d3[1].lo)});
                    if (MODE == XM_DIVQ && pp)
                        bv = df_add2(bv, df2{make_float2(dq[0].hi, dq[1].hi), make_float2(dq[0].lo, dq[1].lo)});
                    const bool u0 = act && live[0], u1 = act && live[1];
                    const float2 val = p2mul(p2add(bv.hi, bv.lo), make_float2(scale, scale));
                    if (u0) {
                        vmax = fmaxf(vmax, fabsf(bv.hi.x));
                        w.bdf[G.cell_off + pbase + (j0 + jl0) * nx + i] = make_float2(bv.hi.x, bv.lo.x);
                    }
                    if (u1) {
                        vmax = fmaxf(vmax, fabsf(bv.hi.y));
                        w.bdf[G.cell_off + pbase + (j0 + jl0 + 1) * nx + i] = make_float2(bv.hi.y, bv.lo.y);
                    }
                    const df2 z = {make_float2(0.f, 0.f), make_float2(0.f, 0.f)};
                    acc2 = df_add2(acc2, df2{make_float2(u0 ? bv.hi.x : z.hi.x, u1 ? bv.hi.y : z.hi.y),
                                             make_float2(u0 ? bv.lo.x : z.lo.x, u1 ? bv.lo.y : z.lo.y)});
                    if (act) {
                        const float v0 = u0 ? val.x : 0.f, v1 = u1 ? val.y : 0.f;
                        float *slot = reinterpret_cast<float *>(buf + (jl0 >> 1) * sstride + spos);
                        if ((jl0 & 1) == 0 && jl0 + 1 < sm.r1) {
                            *reinterpret_cast<float2 *>(slot) = make_float2(v0, v1);
                        } else {
                            slot[jl0 & 1] = v0;
                            if (jl0 + 1 < sm.r1)
                                *(reinterpret_cast<float *>(buf + ((jl0 + 1) >> 1) * sstride + spos) + ((jl0 + 1) & 1)) = v1;
                        }
                    }
                }
                } else {
#pragma unroll
                for (int q = 0; q < kRowGroup; ++q) {
                    const int jl = jg + q, j = j0 + jl;
                    if (jl >= sm.r1) break;  // warp-uniform
                    T val = (T)0;
                    if (j < ny) {
                        const int row = j * nx;
                        V bv;
                        if constexpr (IsDF<A>::value && DIVL) {
                            // the three face differences in fp64 (three DADD per cell, each
                            // rounded to 2^-53 of the difference), then the coefficient
                            // products and their sum in float-float
                            double Un = __shfl_down_sync(0xffffffffu, ru[q], 1);
                            if (own_up) Un = rue[q];
                            const double Vc = vcur64;
                            vcur64 = rvn[q];
                            bv = df_dot3(cu, f64_to_df(__dsub_rn(Un, ru[q])), cv, f64_to_df(__dsub_rn(rvn[q], Vc)),
                                         cwp, f64_to_df(__dsub_rn(rw1[q], rw0[q])));
                            if (MODE == XM_DIVQ && pp) bv = A::add(bv, A::mul(cp, A::load(rp[q])));
                        } else {
                        V U = A::load(ru[q]);
                        V Un = shdown(U, 1);
                        if (own_up) Un = A::load(rue[q]);
                        V Vn = A::load(rvn[q]);
                        const V W0 = A::load(rw0[q]), W1 = A::load(rw1[q]);
                        V Vc = vcur;
                        vcur = Vn;
                        if (MODE == XM_ADJ) {
                            if (zero_u) U = A::zero();
                            if (zero_un) Un = A::zero();
                            if (wall_y && j == 0) Vc = A::zero();
                            if (wall_y && j + 1 == ny) Vn = A::zero();
                        }
                        bv = A::add(A::mul(cu, A::sub(Un, U)), A::mul(cv, A::sub(Vn, Vc)));
                        if (DIVL) {
                            bv = A::add(bv, A::mul(cwp, A::sub(W1, W0)));
                            if (MODE == XM_DIVQ && pp) bv = A::add(bv, A::mul(cp, A::load(rp[q])));
                        } else {
                            bv = A::add(bv, A::sub(A::mul(cwp, W1), A::mul(cwm, W0)));
                            if (pp) bv = A::add(bv, A::mul(cp, A::load(rp[q])));
                        }
                        }
                        have_v = true;
                        if (act) {
                            if (DIVL) vmax = fmaxf(vmax, absv<A>(bv));
                            if constexpr (sizeof(T) == 4)
                                w.bdf[G.cell_off + pbase + row + i] = *reinterpret_cast<const float2 *>(&bv);
                            else if (DIVL && w.bws)
                                w.bws[G.cell_off + pbase + row + i] = *reinterpret_cast<const double *>(&bv);
                            acc = A::add(acc, bv);
                            val = to_T<T, A>(bv) * scale;
                        }
                    } else {
                        have_v = false;
                    }
                    if (act) *(reinterpret_cast<T *>(buf + (jl >> 1) * sstride + spos) + (jl & 1)) = val;
                }
                }
            }
            if constexpr (IsDF<A>::value && DIVL)
                acc = df_add(acc, df_add(df{acc2.hi.x, acc2.lo.x}, df{acc2.hi.y, acc2.lo.y}));
        } else if constexpr (MODE == XM_RESID0 && IsDF<A>::value) {
            // first refinement sweep: phi_0 is plain fp32, so the second differences are
            // exact float sums (a missing wall neighbour is replaced by the cell itself,
            // which zeroes its difference) and only the coefficient products and the
            // final sums round, at float-float precision.
            constexpr int NF = 1;
            constexpr int RG = NF == 2 ? 2 : kRowGroup;  // rows whose loads go together
            const float *phw[2] = {w.phi_hi + G.cell_off + pbase, w.phi_lo + G.cell_off + pbase};
            const float2 *bd = w.bdf + G.cell_off + pbase;
            float Pm[NF], Pc[NF];
#pragma unroll
            for (int f = 0; f < NF; ++f) Pm[f] = Pc[f] = 0.f;
            bool have = false;
            df2 acc2 = {make_float2(0.f, 0.f), make_float2(0.f, 0.f)};  // plane sum of phi, per lane
            df2 accr = {make_float2(0.f, 0.f), make_float2(0.f, 0.f)};  // plane sum of the residual, per lane
            for (int jg = sm.r0; jg < sm.r1; jg += RG) {
                float pn[NF][RG], pkp[NF][RG], pkm[NF][RG], peu[NF][RG], ped[NF][RG];
                float2 bdv[RG];
                float pm0[NF], pc0[NF];
                const bool need0 = !have;
#pragma unroll
                for (int q = 0; q < RG; ++q) {
                    const int jl = jg + q, j = j0 + jl;
#pragma unroll
                    for (int f = 0; f < NF; ++f) {
                        pn[f][q] = pkp[f][q] = pkm[f][q] = peu[f][q] = ped[f][q] = 0.f;
                        if (q == 0) pm0[f] = pc0[f] = 0.f;
                    }
                    bdv[q] = make_float2(0.f, 0.f);
                    if (jl < sm.r1 && j < ny) {
                        const int jp = (j + 1 == ny) ? 0 : j + 1;
                        const int jm = (j == 0) ? ny - 1 : j - 1;
                        const int row = j * nx;
#pragma unroll
                        for (int f = 0; f < NF; ++f) {
                            const float *ph = phw[f];
                            if (q == 0 && need0) {
                                pm0[f] = __ldg(ph + jm * nx + ii);
                                pc0[f] = __ldg(ph + row + ii);
                            }
                            pn[f][q] = __ldg(ph + jp * nx + ii);
                            if (k + 1 < nz) pkp[f][q] = __ldg(ph + plane + row + ii);
                            if (k > 0) pkm[f][q] = __ldg(ph + row + ii - plane);
                            if (own_up) peu[f][q] = __ldg(ph + row + ip);
                            if (own_dn) ped[f][q] = __ldg(ph + row + im);
                        }
                        if (act) bdv[q] = __ldg(bd + row + i);
                    }
                }
                if (need0) {
#pragma unroll
                    for (int f = 0; f < NF; ++f) {
                        Pm[f] = pm0[f];
                        Pc[f] = pc0[f];
                    }
                }
                // two rows at a time: their stencil neighbours gathered as scalars, then the
                // residual of both in two-lane float-float operations (bit for bit the
                // scalar sequence); both rows' values go to one FFT slot (x: even row, y: odd)
#pragma unroll
                for (int q = 0; q < RG; q += 2) {
                    const int jl0 = jg + q;
                    if (jl0 >= sm.r1) break;  // warp-uniform
                    float xp[NF][2], xm[NF][2], yp[NF][2], ym[NF][2], zp[NF][2], zm[NF][2], pc[NF][2];
                    bool live[2];
#pragma unroll
                    for (int h = 0; h < 2; ++h) {
                        const int j = j0 + jl0 + h;
                        live[h] = jl0 + h < sm.r1 && j < ny;
#pragma unroll
                        for (int f = 0; f < NF; ++f) {
                            const float P = Pc[f];
                            float Pip = __shfl_down_sync(0xffffffffu, P, 1);
                            if (own_up) Pip = peu[f][q + h];
                            float Pim = __shfl_up_sync(0xffffffffu, P, 1);
                            if (own_dn) Pim = ped[f][q + h];
                            if (wall_x && ii + 1 == nx) Pip = P;
                            if (wall_x && ii == 0) Pim = P;
                            float Pjp = pn[f][q + h], Pjm = Pm[f];
                            if (wall_y && j + 1 == ny) Pjp = P;
                            if (wall_y && j == 0) Pjm = P;
                            xp[f][h] = Pip; xm[f][h] = Pim; yp[f][h] = Pjp; ym[f][h] = Pjm; pc[f][h] = P;
                            // top: Neumann (difference zero) or Dirichlet outlet (phi = 0 on the face)
                            zp[f][h] = (k + 1 < nz) ? pkp[f][q + h] : (G.dir_top ? 0.f : P);
                            zm[f][h] = (k > 0) ? pkm[f][q + h] : P;
                            if (live[h]) {
                                Pm[f] = P;
                                Pc[f] = pn[f][q + h];
                            }
                        }
                        have = live[h];
                    }
                    df2 d2x, d2y, dzp, dzm;
#pragma unroll
                    for (int f = 0; f < NF; ++f) {
                        const float2 PC = make_float2(pc[f][0], pc[f][1]);
                        const float2 NPC = p2mul(PC, make_float2(-1.f, -1.f)), M2 = p2add(NPC, NPC);
                        const float2 XP = make_float2(xp[f][0], xp[f][1]), XM = make_float2(xm[f][0], xm[f][1]);
                        const float2 YP = make_float2(yp[f][0], yp[f][1]), YM = make_float2(ym[f][0], ym[f][1]);
                        const df2 ax = sum3u2(XP, XM, M2);
                        const df2 ay = sum3u2(YP, YM, M2);
                        const df2 azp = two_sum2(make_float2(zp[f][0], zp[f][1]), NPC);
                        const df2 azm = two_sum2(PC, p2mul(make_float2(zm[f][0], zm[f][1]), make_float2(-1.f, -1.f)));
                        if (f == 0) {
                            d2x = ax; d2y = ay; dzp = azp; dzm = azm;
                        } else {
                            d2x = df_add2(d2x, ax); d2y = df_add2(d2y, ay);
                            dzp = df_add2(dzp, azp); dzm = df_add2(dzm, azm);
                        }
                    }
                    const df2 bv2 = {make_float2(bdv[q].x, bdv[q + 1].x), make_float2(bdv[q].y, bdv[q + 1].y)};
                    const df2 r = df_resid4_2(bv2, cp, cu, d2x, cv, d2y, cwp, dzp, cwm, dzm);
                    const float2 val = p2mul(p2add(r.hi, r.lo), make_float2(scale, scale));
                    const bool u0 = act && live[0], u1 = act && live[1];
                    if (w.rdf) {  // two or more sweeps: the second starts from this residual
                        float2 *rd = w.rdf + G.cell_off + pbase + (j0 + jl0) * nx + i;
                        if (u0) rd[0] = make_float2(r.hi.x, r.lo.x);
                        if (u1) rd[nx] = make_float2(r.hi.y, r.lo.y);
                    }
#pragma unroll
                    for (int f = 0; f < NF; ++f)
                        acc2 = df_addf2(acc2, make_float2(u0 ? pc[f][0] : 0.f, u1 ? pc[f][1] : 0.f));
                    accr = df_add2(accr, df2{make_float2(u0 ? r.hi.x : 0.f, u1 ? r.hi.y : 0.f),
                                             make_float2(u0 ? r.lo.x : 0.f, u1 ? r.lo.y : 0.f)});
                    if (act) {
                        const float v0 = u0 ? val.x : 0.f, v1 = u1 ? val.y : 0.f;
                        float *slot = reinterpret_cast<float *>(buf + (jl0 >> 1) * sstride + spos);
                        if ((jl0 & 1) == 0 && jl0 + 1 < sm.r1) {
                            *reinterpret_cast<float2 *>(slot) = make_float2(v0, v1);
                        } else {
                            slot[jl0 & 1] = v0;
                            if (jl0 + 1 < sm.r1)
                                *(reinterpret_cast<float *>(buf + ((jl0 + 1) >> 1) * sstride + spos) + ((jl0 + 1) & 1)) = v1;
                        }
                    }
                }
            }
            acc_phi = df_add(acc_phi, df_add(df{acc2.hi.x, acc2.lo.x}, df{acc2.hi.y, acc2.lo.y}));
            acc = df_add(acc, df_add(df{accr.hi.x, accr.lo.x}, df{accr.hi.y, accr.lo.y}));
        } else if constexpr (MODE == XM_RESID1 && IsDF<A>::value) {
            // second refinement sweep: phi = phi_0 + delta_1 (hi, lo), and the first sweep's
            // residual r_1 = b - <b> - L phi_0 is kept per cell, so r_2 = r_1 - L delta_1.
            // delta_1's first differences are rounded to fp32 exactly as the velocity
            // correction rounds the trailing words' differences (df_sub_acc), so that this
            // rounding cancels in D u; the second differences of those floats are exact
            // float-float pairs, then products and sums as in the first sweep, two rows at
            // a time.  phi_0 is read at the cell only, for the plane sums of phi.
            const float *dl = w.phi_lo + G.cell_off + pbase, *p0 = w.phi_hi + G.cell_off + pbase;
            const float2 *rd = w.rdf + G.cell_off + pbase;
            constexpr int RG = kRowGroup;
            float Dm = 0.f, Dc = 0.f;
            bool have = false;
            df2 acc2 = {make_float2(0.f, 0.f), make_float2(0.f, 0.f)};  // plane sum of phi, per lane
            df2 accr = {make_float2(0.f, 0.f), make_float2(0.f, 0.f)};  // plane sum of the residual, per lane
            for (int jg = sm.r0; jg < sm.r1; jg += RG) {
                float pn[RG], pkp[RG], pkm[RG], peu[RG], ped[RG], ph0[RG];
                float2 rv[RG];
                float pm0 = 0.f, pc0 = 0.f;
                const bool need0 = !have;
#pragma unroll
                for (int q = 0; q < RG; ++q) {
                    const int jl = jg + q, j = j0 + jl;
                    pn[q] = pkp[q] = pkm[q] = peu[q] = ped[q] = ph0[q] = 0.f;
                    rv[q] = make_float2(0.f, 0.f);
                    if (jl < sm.r1 && j < ny) {
                        const int jp = (j + 1 == ny) ? 0 : j + 1;
                        const int jm = (j == 0) ? ny - 1 : j - 1;
                        const int row = j * nx;
                        if (q == 0 && need0) {
                            pm0 = __ldg(dl + jm * nx + ii);
                            pc0 = __ldg(dl + row + ii);
                        }
                        pn[q] = __ldg(dl + jp * nx + ii);
                        if (k + 1 < nz) pkp[q] = __ldg(dl + plane + row + ii);
                        if (k > 0) pkm[q] = __ldg(dl + row + ii - plane);
                        if (own_up) peu[q] = __ldg(dl + row + ip);
                        if (own_dn) ped[q] = __ldg(dl + row + im);
                        if (act) {
                            rv[q] = __ldg(rd + row + i);
                            ph0[q] = __ldg(p0 + row + i);
                        }
                    }
                }
                if (need0) {
                    Dm = pm0;
                    Dc = pc0;
                }
#pragma unroll
                for (int q = 0; q < RG; q += 2) {
                    const int jl0 = jg + q;
                    if (jl0 >= sm.r1) break;  // warp-uniform
                    float xp[2], xm[2], yp[2], ym[2], zp[2], zm[2], pc[2];
                    bool live[2];
#pragma unroll
                    for (int h = 0; h < 2; ++h) {
                        const int j = j0 + jl0 + h;
                        live[h] = jl0 + h < sm.r1 && j < ny;
                        const float P = Dc;
                        float Pip = __shfl_down_sync(0xffffffffu, P, 1);
                        if (own_up) Pip = peu[q + h];
                        float Pim = __shfl_up_sync(0xffffffffu, P, 1);
                        if (own_dn) Pim = ped[q + h];
                        // wall faces carry no gradient: the neighbour is the cell itself
                        if (wall_x && ii + 1 == nx) Pip = P;
                        if (wall_x && ii == 0) Pim = P;
                        float Pjp = pn[q + h], Pjm = Dm;
                        if (wall_y && j + 1 == ny) Pjp = P;
                        if (wall_y && j == 0) Pjm = P;
                        xp[h] = Pip; xm[h] = Pim; yp[h] = Pjp; ym[h] = Pjm; pc[h] = P;
                        // top: Neumann (difference zero) or Dirichlet outlet (phi = 0 on the face)
                        zp[h] = (k + 1 < nz) ? pkp[q + h] : (G.dir_top ? 0.f : P);
                        zm[h] = (k > 0) ? pkm[q + h] : P;
                        if (live[h]) {
                            Dm = P;
                            Dc = pn[q + h];
                        }
                        have = live[h];
                    }
                    const float2 PC = make_float2(pc[0], pc[1]);
                    // first differences rounded to fp32 (the correction's fl(lo_a - lo_b)),
                    // second differences exact
                    const float2 fxp = p2sub(make_float2(xp[0], xp[1]), PC), fxm = p2sub(PC, make_float2(xm[0], xm[1]));
                    const float2 fyp = p2sub(make_float2(yp[0], yp[1]), PC), fym = p2sub(PC, make_float2(ym[0], ym[1]));
                    const df2 d2x = two_sum2(fxp, p2mul(fxm, make_float2(-1.f, -1.f)));
                    const df2 d2y = two_sum2(fyp, p2mul(fym, make_float2(-1.f, -1.f)));
                    const df2 dzp = {p2sub(make_float2(zp[0], zp[1]), PC), make_float2(0.f, 0.f)};
                    const df2 dzm = {p2sub(PC, make_float2(zm[0], zm[1])), make_float2(0.f, 0.f)};
                    const df2 r1 = {make_float2(rv[q].x, rv[q + 1].x), make_float2(rv[q].y, rv[q + 1].y)};
                    const df zero = {0.f, 0.f};
                    const df2 r = df_resid4_2(r1, zero, cu, d2x, cv, d2y, cwp, dzp, cwm, dzm);
                    const float2 val = p2mul(p2add(r.hi, r.lo), make_float2(scale, scale));
                    const bool u0 = act && live[0], u1 = act && live[1];
                    acc2 = df_addf2(acc2, make_float2(u0 ? ph0[q] : 0.f, u1 ? ph0[q + 1] : 0.f));
                    acc2 = df_addf2(acc2, make_float2(u0 ? pc[0] : 0.f, u1 ? pc[1] : 0.f));
                    accr = df_add2(accr, df2{make_float2(u0 ? r.hi.x : 0.f, u1 ? r.hi.y : 0.f),
                                             make_float2(u0 ? r.lo.x : 0.f, u1 ? r.lo.y : 0.f)});
                    if (act) {
                        const float v0 = u0 ? val.x : 0.f, v1 = u1 ? val.y : 0.f;
                        float *slot = reinterpret_cast<float *>(buf + (jl0 >> 1) * sstride + spos);
                        if ((jl0 & 1) == 0 && jl0 + 1 < sm.r1) {
                            *reinterpret_cast<float2 *>(slot) = make_float2(v0, v1);
                        } else {
                            slot[jl0 & 1] = v0;
                            if (jl0 + 1 < sm.r1)
                                *(reinterpret_cast<float *>(buf + ((jl0 + 1) >> 1) * sstride + spos) + ((jl0 + 1) & 1)) = v1;
                        }
                    }
                }
            }
            acc_phi = df_add(acc_phi, df_add(df{acc2.hi.x, acc2.lo.x}, df{acc2.hi.y, acc2.lo.y}));
            acc = df_add(acc, df_add(df{accr.hi.x, accr.lo.x}, df{accr.hi.y, accr.lo.y}));
        } else if constexpr (MODE == XM_RESID && IsDF<A>::value) {
            // a later refinement sweep (the third and after; the second is XM_RESID1 where
            // the first sweep's residual is kept): phi = hi + lo (float-float, possibly
            // unnormalised).  The first differences of phi are formed exactly as the velocity
            // correction forms them (df_sub_acc, lane for lane), so that their one fp32
            // rounding is part of the residual this sweep corrects and cancels in D u; second
            // differences, products and sums as in the first sweep, two rows at a time in
            // packed operations.
            const float *phw[2] = {w.phi_hi + G.cell_off + pbase, w.phi_lo + G.cell_off + pbase};
            const float2 *bd = w.bdf + G.cell_off + pbase;
            float Pm[2] = {0.f, 0.f}, Pc[2] = {0.f, 0.f};
            bool have = false;
            df2 acc2 = {make_float2(0.f, 0.f), make_float2(0.f, 0.f)};  // plane sum of phi, per lane
            df2 accr = {make_float2(0.f, 0.f), make_float2(0.f, 0.f)};  // plane sum of the residual, per lane
            constexpr int RG = 2;
            for (int jg = sm.r0; jg < sm.r1; jg += RG) {
                float pn[2][RG], pkp[2][RG], pkm[2][RG], peu[2][RG], ped[2][RG];
                float2 bdv[RG];
                float pm0[2] = {0.f, 0.f}, pc0[2] = {0.f, 0.f};
                const bool need0 = !have;
#pragma unroll
                for (int q = 0; q < RG; ++q) {
                    const int jl = jg + q, j = j0 + jl;
#pragma unroll
                    for (int f = 0; f < 2; ++f) pn[f][q] = pkp[f][q] = pkm[f][q] = peu[f][q] = ped[f][q] = 0.f;
                    bdv[q] = make_float2(0.f, 0.f);
                    if (jl < sm.r1 && j < ny) {
                        const int jp = (j + 1 == ny) ? 0 : j + 1;
                        const int jm = (j == 0) ? ny - 1 : j - 1;
                        const int row = j * nx;
#pragma unroll
                        for (int f = 0; f < 2; ++f) {
                            const float *ph = phw[f];
                            if (q == 0 && need0) {
                                pm0[f] = __ldg(ph + jm * nx + ii);
                                pc0[f] = __ldg(ph + row + ii);
                            }
                            pn[f][q] = __ldg(ph + jp * nx + ii);
                            if (k + 1 < nz) pkp[f][q] = __ldg(ph + plane + row + ii);
                            if (k > 0) pkm[f][q] = __ldg(ph + row + ii - plane);
                            if (own_up) peu[f][q] = __ldg(ph + row + ip);
                            if (own_dn) ped[f][q] = __ldg(ph + row + im);
                        }
                        if (act) bdv[q] = __ldg(bd + row + i);
                    }
                }
                if (need0) {
#pragma unroll
                    for (int f = 0; f < 2; ++f) {
                        Pm[f] = pm0[f];
                        Pc[f] = pc0[f];
                    }
                }
                const int jl0 = jg;
                if (jl0 >= sm.r1) break;  // warp-uniform
                // the two rows' stencil values as float-float pairs, lanes = rows
                float xp[2][2], xm[2][2], yp[2][2], ym[2][2], zp[2][2], zm[2][2], pc[2][2];
                bool live[2];
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    const int j = j0 + jl0 + h;
                    live[h] = jl0 + h < sm.r1 && j < ny;
#pragma unroll
                    for (int f = 0; f < 2; ++f) {
                        const float P = Pc[f];
                        float Pip = __shfl_down_sync(0xffffffffu, P, 1);
                        if (own_up) Pip = peu[f][h];
                        float Pim = __shfl_up_sync(0xffffffffu, P, 1);
                        if (own_dn) Pim = ped[f][h];
                        // wall faces carry no gradient: the neighbour is the cell itself,
                        // whose difference df_sub makes exactly zero
                        if (wall_x && ii + 1 == nx) Pip = P;
                        if (wall_x && ii == 0) Pim = P;
                        float Pjp = pn[f][h], Pjm = Pm[f];
                        if (wall_y && j + 1 == ny) Pjp = P;
                        if (wall_y && j == 0) Pjm = P;
                        xp[f][h] = Pip; xm[f][h] = Pim; yp[f][h] = Pjp; ym[f][h] = Pjm; pc[f][h] = P;
                        // top: Neumann (difference zero) or Dirichlet outlet (phi = 0 on the face)
                        zp[f][h] = (k + 1 < nz) ? pkp[f][h] : (G.dir_top ? 0.f : P);
                        zm[f][h] = (k > 0) ? pkm[f][h] : P;
                        if (live[h]) {
                            Pm[f] = P;
                            Pc[f] = pn[f][h];
                        }
                    }
                    have = live[h];
                }
                auto pair = [](const float (&a)[2][2]) {
                    return df2{make_float2(a[0][0], a[0][1]), make_float2(a[1][0], a[1][1])};
                };
                const df2 PC = pair(pc);
                const df2 d2x = df_sub2(df_sub2_acc(pair(xp), PC), df_sub2_acc(PC, pair(xm)));
                const df2 d2y = df_sub2(df_sub2_acc(pair(yp), PC), df_sub2_acc(PC, pair(ym)));
                const df2 dzp = df_sub2_acc(pair(zp), PC);
                const df2 dzm = df_sub2_acc(PC, pair(zm));
                const df2 bv2 = {make_float2(bdv[0].x, bdv[1].x), make_float2(bdv[0].y, bdv[1].y)};
                const df2 r = df_resid4_2(bv2, cp, cu, d2x, cv, d2y, cwp, dzp, cwm, dzm);
                const float2 val = p2mul(p2add(r.hi, r.lo), make_float2(scale, scale));
                const bool u0 = act && live[0], u1 = act && live[1];
                acc2 = df_addf2(acc2, make_float2(u0 ? pc[0][0] : 0.f, u1 ? pc[0][1] : 0.f));
                acc2 = df_addf2(acc2, make_float2(u0 ? pc[1][0] : 0.f, u1 ? pc[1][1] : 0.f));
                accr = df_add2(accr, df2{make_float2(u0 ? r.hi.x : 0.f, u1 ? r.hi.y : 0.f),
                                         make_float2(u0 ? r.lo.x : 0.f, u1 ? r.lo.y : 0.f)});
                if (act) {
                    const float v0 = u0 ? val.x : 0.f, v1 = u1 ? val.y : 0.f;
                    float *slot = reinterpret_cast<float *>(buf + (jl0 >> 1) * sstride + spos);
                    if ((jl0 & 1) == 0 && jl0 + 1 < sm.r1) {
                        *reinterpret_cast<float2 *>(slot) = make_float2(v0, v1);
                    } else {
                        slot[jl0 & 1] = v0;
                        if (jl0 + 1 < sm.r1)
                            *(reinterpret_cast<float *>(buf + ((jl0 + 1) >> 1) * sstride + spos) + ((jl0 + 1) & 1)) = v1;
                    }
                }
            }
            acc_phi = df_add(acc_phi, df_add(df{acc2.hi.x, acc2.lo.x}, df{acc2.hi.y, acc2.lo.y}));
            acc = df_add(acc, df_add(df{accr.hi.x, accr.lo.x}, df{accr.hi.y, accr.lo.y}));
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
                        const V dzp = (k + 1 < nz) ? A::sub(pkp[q], Pc) : (G.dir_top ? A::sub(A::zero(), Pc) : A::zero());
                        const V dzm = (k > 0) ? A::sub(Pc, pkm[q]) : A::zero();
                        // wall faces carry no gradient (Neumann phi)
                        const V dxp = (wall_x && ii + 1 == nx) ? A::zero() : A::sub(Pip, Pc);
                        const V dxm = (wall_x && ii == 0) ? A::zero() : A::sub(Pc, Pim);
                        const V dyp = (wall_y && j + 1 == ny) ? A::zero() : A::sub(pn[q], Pc);
                        const V dym = (wall_y && j == 0) ? A::zero() : A::sub(Pc, Pm);
                        V lap = A::add(A::mul(cu, A::sub(dxp, dxm)), A::mul(cv, A::sub(dyp, dym)));
                        lap = A::add(lap, A::sub(A::mul(cwp, dzp), A::mul(cwm, dzm)));
                        if (act) {
                            V bvv = A::zero();
                            if constexpr (sizeof(T) == 4) bvv = df{bdv[q].x, bdv[q].y};
                            const V bv = A::sub(A::sub(bvv, cp), lap);
                            acc_phi = A::add(acc_phi, Pc);
                            acc = A::add(acc, bv);
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
    // plane sums of this block's rows (for the singular mode), fixed reduction order:
    // of the right-hand side in the first pass; of the residual and of phi in a
    // refinement pass.  k_00 takes the (0,0) mode of the correction from the residual's
    // plane means (small once phi is close, so their rounding is small too) and the
    // weighted mean of phi from phi's.  With the split, a slot per half row block.
    const int pslot = G.part_off + (k * nrb + rb) * SPLIT + half;
    if (MODE != XM_COPY) {
        V tot = Red<A>::sum(acc, red);
        if (threadIdx.x == 0) w.partial[pslot] = A::store_once(tot);
    }
    if (MODE == XM_RESID || MODE == XM_RESID0 || MODE == XM_RESID1) {
        V totp = Red<A>::sum(acc_phi, red);
        if (threadIdx.x == 0) w.partial_phi[pslot] = A::store_once(totp);
    }
    if (DIVL) {
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
    const FDiv fmb = G.fmb, frows = SPLIT == 2 ? G.fnpair : G.frows;  // fnpair: rows / 2
    if (sizeof(T) == 4 && mb == 1 && !wall_x && ((G.spec_off | ny | j0) & 1) == 0 &&
        (kXThreads / SPLIT) % (rows >> 1) == 0) {
        // one x-mode per column block: every thread keeps one row pair (one packed
        // sequence, rows 2s and 2s + 1, adjacent in the spectrum of a mode) and steps through
        // the modes; the pair's two values come from the same Z_m and Z_{nx-m} and leave as
        // one 16-byte store
        const int npair = rows >> 1;
        const FDiv fnp = SPLIT == 2 ? G.fnpair2 : G.fnpair;
        const int m0 = (int)fdiv((unsigned)threadIdx.x, fnp), mstep = (kXThreads / SPLIT) / npair;
        const int s_ = threadIdx.x - m0 * npair, ja = j0 + 2 * s_;
        if (ja < ny) {  // ny even: row ja + 1 exists with row ja
            const cx<T> *seq = buf + s_ * sstride;
            float4 *dst = reinterpret_cast<float4 *>(spec + ja);
            for (int m = m0; m < nxh; m += mstep) {
                const cx<T> Zm = seq[pos_tr(m, N1, N2, fN1)];
                const cx<T> Zc = seq[pos_tr(m == 0 ? 0 : nx - m, N1, N2, fN1)];
                dst[(size_t)m * (ny >> 1)] = make_float4((Zm.x + Zc.x) * 0.5f, (Zm.y - Zc.y) * 0.5f,
                                                         (Zm.y + Zc.y) * 0.5f, (Zc.x - Zm.x) * 0.5f);
            }
        }
        return;
    }
    if (mb == 1 && (kXThreads / SPLIT) % rows == 0 && !wall_x) {
        // one x-mode per column block: every thread keeps one row jl and steps through
        // the modes m0, m0 + blockDim / rows, ... (the rows of one mode are contiguous
        // in the spectrum, so consecutive threads store consecutive elements)
        const int m0 = (int)fdiv((unsigned)threadIdx.x, frows), mstep = (kXThreads / SPLIT) / rows;
        const int jl = threadIdx.x - m0 * rows, j = j0 + jl;
        if (j < ny) {
            const cx<T> *seq = buf + (jl >> 1) * sstride;
            cx<T> *dst = spec + j;
            const bool odd = (jl & 1) != 0;
            for (int m = m0; m < nxh; m += mstep) {
                const cx<T> Zm = seq[pos_tr(m, N1, N2, fN1)];
                const cx<T> Zc = seq[pos_tr(m == 0 ? 0 : nx - m, N1, N2, fN1)];
                const cx<T> X = odd ? cx<T>{(Zm.y + Zc.y) * (T)0.5, (Zc.x - Zm.x) * (T)0.5}
                                    : cx<T>{(Zm.x + Zc.x) * (T)0.5, (Zm.y - Zc.y) * (T)0.5};
                dst[(size_t)m * ny] = X;
            }
        }
        return;
    }
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
        if (wall_x) {  // DCT-II coefficient m = Re(exp(-i pi m/(2 nx)) X_m), kept as (c, 0)
            const cx<T> tw = twx[G.dctx_off - G.twx_off + m];
            X = {tw.x * X.x - tw.y * X.y, (T)0};
        }
        spec[((size_t)cb * ny + j) * mb + mm] = X;
    }
}

// ================================================================ k_xinv
// Inverse real FFT along x of a block of rows; STORE writes phi (fp64 path: fp64
// array; mixed path: the hi array of the float-float phi), ACCUM adds the
// refinement correction to the float-float phi.
// SPLIT = 2: two CTAs of kXThreads / 2 threads per row block, each transforming half
// of its rows (every grid of the plan has rows divisible by 4): twice the CTAs per SM
// at the same warp count, so that one CTA's FFT overlaps another's gather and store;
// five of them per SM (96 registers).
template <typename T, class A, int IMODE, bool W, int SPLIT>
__global__ void __launch_bounds__(kXThreads / SPLIT, SPLIT == 2 ? 5 : (sizeof(T) == 4 ? 2 : 1))
    k_xinv(Work w, UserPtrs p, int use_ws, int lo_valid) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    cx<T> *buf = reinterpret_cast<cx<T> *>(smem_raw);
    const int b = blockIdx.x / SPLIT + p.blk0;
    const int half = SPLIT == 2 ? (int)(blockIdx.x & 1u) : 0;
    const int g = find_grid(w.xblk_start, w.ngrids, b);
    const GridDev &G = w.grids[g];
    const int lb = b - __ldg(w.xblk_start + g);
    const int nrb = G.nrb, rows = G.rows / SPLIT;
    const int k = lb / nrb, rb = lb - k * nrb;
    const int j0 = rb * G.rows + half * rows;
    const int nx = G.nx, ny = G.ny;
    // sequences one complex element further apart than their length, so that the
    // split / gather steps, which read the same position of several sequences, do not
    // fall into one shared-memory bank
    const int N1 = G.nx1, N2 = G.nx2, sstride = fft_seq_len(N1, N2) + 1;
    const FDiv fN1 = G.fnx1, fN2 = G.fnx2, fmb = G.fmb, fnpair = SPLIT == 2 ? G.fnpair2 : G.fnpair, fnx = G.fnx;
    const int mb = G.mb, ncb = G.ncb, nxh = G.nxh;
    const cx<T> *spec = reinterpret_cast<const cx<T> *>(w.spec) + G.spec_off + (size_t)k * ncb * ny * mb;
    const cx<T> *twx = reinterpret_cast<const cx<T> *>(w.twx) + G.twx_off;
    const int npair = rows >> 1;
    const int nload = ncb * npair * mb;
    if (sizeof(T) == 4 && !(W && G.wall_x) && mb == 1 && ((G.spec_off | ny | j0) & 1) == 0) {
        // one x-mode per column block (the spectrum of mode m is a run of ny values): the
        // row pair's two values A_m, B_m are adjacent, so one 16-byte load brings both and
        // the packed FFT input is formed on the spot, Z_m = A_m + i B_m and
        // Z_{nx-m} = conj(A_m) + i conj(B_m), with no staging pass
        // (kGatherBatch loads in flight per thread before any of them is used)
        constexpr int kGatherBatch = 8;
        const int nt = npair * nxh, nthr = blockDim.x;
        for (int t0 = threadIdx.x; t0 < nt; t0 += kGatherBatch * nthr) {
            float4 v[kGatherBatch];
            int mq[kGatherBatch], sq[kGatherBatch];
#pragma unroll
            for (int u = 0; u < kGatherBatch; ++u) {
                const int t = t0 + u * nthr;
                v[u] = make_float4(0.f, 0.f, 0.f, 0.f);
                mq[u] = -1;
                sq[u] = 0;
                if (t < nt) {
                    const int m = (int)fdiv((unsigned)t, fnpair);
                    const int s_ = t - m * npair;
                    const int ja = j0 + 2 * s_;  // even, and ny is even: row ja + 1 exists with row ja
                    mq[u] = m;
                    sq[u] = s_;
                    if (ja < ny) v[u] = __ldg(reinterpret_cast<const float4 *>(spec + (size_t)m * ny + ja));
                }
            }
#pragma unroll
            for (int u = 0; u < kGatherBatch; ++u) {
                const int m = mq[u];
                if (m < 0) continue;
                cx<T> *seq = buf + sq[u] * sstride;
                seq[pos_tr(m, N1, N2, fN1)] = {(T)(v[u].x - v[u].w), (T)(v[u].y + v[u].z)};
                if (m != 0 && 2 * m != nx)
                    seq[pos_tr(nx - m, N1, N2, fN1)] = {(T)(v[u].x + v[u].w), (T)(v[u].z - v[u].y)};
            }
        }
    } else if (!(W && G.wall_x)) {
        // real FFT input Z = X_a + i X_b of the row pair (a, b): Z_m = A_m + i B_m and
        // Z_{nx-m} = conj(A_m) + i conj(B_m).  Every spectrum value is first copied
        // asynchronously straight to shared memory (the whole block's input in flight at
        // once): A_m to the slot of Z_m, B_m to the slot of Z_{nx-m}, or, where that is
        // Z_m itself (m = 0, m = nx/2), to a padding slot of the sequence (N2: the pad
        // column of row 0; N1 (N2+1): the pad after the last row).  A pass over the
        // pairs (m, nx-m) then forms Z in place.
        const int seqlen = fft_seq_len(N1, N2);
        for (int t = threadIdx.x; t < nload; t += blockDim.x) {
            const int rest = (int)fdiv((unsigned)t, fmb);
            const int mm = t - rest * mb;
            const int cb = (int)fdiv((unsigned)rest, fnpair);
            const int s_ = rest - cb * npair;
            const int m = cb * mb + mm;
            if (m >= nxh) continue;
            cx<T> *seq = buf + s_ * sstride;
            cx<T> *da = seq + pos_tr(m, N1, N2, fN1);
            cx<T> *db = seq + (m == 0 ? N2 : (2 * m == nx ? seqlen : pos_tr(nx - m, N1, N2, fN1)));
            const int ja = j0 + 2 * s_, jb = ja + 1;
            const cx<T> *src = spec + ((size_t)cb * ny + ja) * mb + mm;
            if (ja < ny) cp_async<sizeof(cx<T>)>(da, src);
            else *da = {(T)0, (T)0};
            if (jb < ny) cp_async<sizeof(cx<T>)>(db, src + mb);
            else *db = {(T)0, (T)0};
        }
        cp_async_commit();
        cp_async_wait<0>();
        __syncthreads();
        const int npm = nx / 2 + 1;  // pairs (m, nx-m), m = 0..nx/2
        const FDiv fnph = G.fnph;
        for (int t = threadIdx.x; t < npair * npm; t += blockDim.x) {
            const int s_ = (int)fdiv((unsigned)t, fnph), m = t - s_ * npm;
            cx<T> *seq = buf + s_ * sstride;
            const int pa = pos_tr(m, N1, N2, fN1);
            const bool self = m == 0 || 2 * m == nx;
            const int pb = m == 0 ? N2 : (2 * m == nx ? seqlen : pos_tr(nx - m, N1, N2, fN1));
            const cx<T> a = seq[pa], bb = seq[pb];
            seq[pa] = {a.x - bb.y, a.y + bb.x};
            if (!self) seq[pb] = {a.x + bb.y, bb.x - a.y};
        }
    } else {
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
        {   // wall-bounded x: DCT-III input stage of two real coefficient rows a, b (real parts of the
            // spectrum): V_m = conj(W^m)(X_m - i X_{N-m}) per row, X_N = 0, packed as
            // V^a + i V^b; the unscaled inverse FFT then yields row a + i row b, reordered.
            T ac = (T)0, bc = (T)0;
            if (m > 0) {
                const int mc = nx - m, cbc = mc / mb, mmc = mc - cbc * mb;
                if (ja < ny) ac = spec[((size_t)cbc * ny + ja) * mb + mmc].x;
                if (jb < ny) bc = spec[((size_t)cbc * ny + jb) * mb + mmc].x;
            }
            const cx<T> tw = twx[G.dctx_off - G.twx_off + m];
            const cx<T> Va = {tw.x * A_.x - tw.y * ac, -tw.x * ac - tw.y * A_.x};
            const cx<T> Vb = {tw.x * B_.x - tw.y * bc, -tw.x * bc - tw.y * B_.x};
            seq[pos_tr(m, N1, N2, fN1)] = {Va.x - Vb.y, Va.y + Vb.x};
        }
    }
    }
    __syncthreads();
    fft_batch<T, +1>(buf, npair, sstride, N1, N2, fN1, fN2, twx);

    const int gi = g - p.g0;
    const ptrdiff_t plane = (ptrdiff_t)nx * ny;
    const ptrdiff_t base = (ptrdiff_t)k * plane + (ptrdiff_t)j0 * nx;
    const int ncell = max(0, min(rows, ny - j0)) * nx;
    double *phi64 = nullptr;
    float *phh = nullptr, *phl = nullptr, *pl2 = nullptr;
    if (sizeof(T) == 8) phi64 = (use_ws ? (w.phi_ws + G.cell_off) : p.out_p[gi]) + base;
    else {
        phh = w.phi_hi + G.cell_off + base;
        phl = w.phi_lo + G.cell_off + base;
        if (IMODE == IM_LAST) pl2 = w.phi_lo2 + G.cell_off + base;
    }
    auto put = [&](int t, T val) {
        if constexpr (sizeof(T) == 8) {
            phi64[t] = (double)val;
        } else {
            if (IMODE == IM_STORE) {
                phh[t] = (float)val;
            } else if (IMODE == IM_LAST) {
                pl2[t] = (float)val;  // phi = hi + lo + lo2, read so by the correction
            } else if (!lo_valid) {
                phl[t] = (float)val;  // phi = phi_0 + delta held as the unevaluated pair (hi, lo)
            } else {
                // (hi, lo) may be unnormalised (lo = the first correction, larger than an
                // ulp of hi): hi + lo + val is formed without error in three floats and
                // rounded once into a normalised pair, so the correction keeps its low bits
                const df nw = df_add3(phh[t], phl[t], (float)val);
                phh[t] = nw.hi;
                phl[t] = nw.lo;
            }
        }
    };
    if (!(W && G.wall_x) && (int)blockDim.x % N2 == 0) {
        // rows outer; along a row the FFT position advances by blockDim + blockDim / N2
        // per step (N2 divides the block size), so the inner loop needs no division
        const int nrow = ncell / nx, pos0 = pos_nat(threadIdx.x, fN2);
        const int pstep = (int)blockDim.x + (int)blockDim.x / N2;
        for (int jl = 0; jl < nrow; ++jl) {
            const cx<T> *seq = buf + (jl >> 1) * sstride;
            const bool odd = (jl & 1) != 0;
            int pos = pos0;
            for (int i = threadIdx.x; i < nx; i += blockDim.x, pos += pstep) {
                const cx<T> z = seq[pos];
                put(jl * nx + i, odd ? z.y : z.x);
            }
        }
        return;
    }
    for (int t = threadIdx.x; t < ncell; t += blockDim.x) {
        const int jl = (int)fdiv((unsigned)t, fnx), i = t - jl * nx;
        const cx<T> z = buf[(jl >> 1) * sstride + pos_nat((W && G.wall_x) ? dct_perm(i, nx) : i, fN2)];
        put(t, (jl & 1) ? z.y : z.x);
    }
}

// ================================================================ k_correct
constexpr int kRowGroupC = 2;

// forward (ADJ = 0): u = u* + s rdx (phi_{i-1} - phi_i), v likewise,
//                    w_k = w*_k + s rgzf_k (phi_{k-1} - phi_k), wall faces copied;
//                    mixed path: also writes phi (fp64) from its float-float value.
// adjoint (ADJ = 1): g* = g_u + hz_k rdx (psi_{i-1} - psi_i), ...,
//                    w_k = g_w,k + psi_{k-1} [k>=1] - psi_k [k<=nz-1].
// PU: forward with a pressure update (pmode 1: p_n + phi, 2: minus cimp (b - <b>)).
// L2 (mixed path, two or more sweeps): phi is hi + lo + lo2, with lo2 the last sweep's
// correction in phi_lo2; its differences are formed in fp32 beside those of the pair (lo2
// is a few 1e-10 of phi, so they round far below the pair's last bit) and added to them.
template <class A, int ADJ, bool W, bool PU, bool L2 = false>
// mixed: five CTAs per SM (48 registers; a few spilled bytes cost less than the fifth
// CTA's latency hiding gains on the loads), four with lo2; fp64: room for the pressure terms
__global__ void __launch_bounds__(kXThreads, IsDF<A>::value ? (L2 ? 4 : 5) : 3)
    k_correct(Work w, UserPtrs p, int use_ws, int lo_valid, double s, int pmode, double cimp) {
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
    const float *l2p = nullptr;  // lo2 of the plane (L2)
    if constexpr (MIX) {
        ph.hi = w.phi_hi + G.cell_off + pbase;
        ph.lo = lo_valid ? w.phi_lo + G.cell_off + pbase : nullptr;
        if (L2) l2p = w.phi_lo2 + G.cell_off + pbase;
    } else {
        ph.p = (use_ws ? (w.phi_ws + G.cell_off) : p.out_p[gi]) + pbase;
    }
    // wall-bounded x: u rows hold nx+1 faces; wall-bounded y: v planes hold ny+1 rows
    const int wall_x = W ? G.wall_x : 0, wall_y = W ? G.wall_y : 0, nxu = W ? G.nxu : nx;
    const ptrdiff_t ubase = (ptrdiff_t)k * ny * nxu, vbase = (ptrdiff_t)k * (W ? G.nyv : ny) * nx;
    const double *ui = p.in_u[gi] + ubase, *vi = p.in_v[gi] + vbase, *wi = p.in_w[gi] + pbase;
    double *uo = p.out_u[gi] + ubase, *vo = p.out_v[gi] + vbase, *wo = p.out_w[gi] + pbase;
    // pressure output (forward): phi (mixed path; the fp64 path's phi is already in out.p),
    // or p_n + phi [- cimp (b - <b>)] (Eq. pressure) with p_n = in.p
    double *po = (!ADJ && (MIX || PU)) ? p.out_p[gi] + pbase : nullptr;
    const double *pn = (!ADJ && PU) ? p.in_p[gi] + pbase : nullptr;
    const double mean_b = PU ? w.mean_b[g] : 0.0;
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
    // outlet face coefficient (rgzf[nz] is 0 unless the top is a Dirichlet outlet)
    const V cwt = Coef<A>::c(ADJ ? 0.0 : s * w.z.rgzf[zo + nz]);
    const int lane = threadIdx.x & 31;
    const SegMap sm = seg_map(nx, rows);
    for (int seg = sm.seg0; seg < sm.nseg; seg += sm.segstep) {
        const int i = seg * 32 + lane;
        const bool act = i < nx;
        const int ii = act ? i : nx - 1;
        const int im = (ii == 0) ? nx - 1 : ii - 1;
        const bool own_dn = (lane == 0) || (ii == 0);
        const bool wall_lo = wall_x && ii == 0;  // face 0 of a wall-bounded row
        V Pjm = A::zero();
        float L2jm = 0.f;
        bool have = false;
        for (int jg = sm.r0; jg < sm.r1; jg += kRowGroupC) {
            V pc[kRowGroupC], pkm[kRowGroupC], ped[kRowGroupC];
            float lc[kRowGroupC], lkm[kRowGroupC], led[kRowGroupC];  // lo2 (L2)
            double ru[kRowGroupC], rv[kRowGroupC], rw[kRowGroupC], rwt[kRowGroupC];
            V pjm0 = A::zero();
            float ljm0 = 0.f;
            const bool need0 = !have;
#pragma unroll
            for (int q = 0; q < kRowGroupC; ++q) {
                const int jl = jg + q, j = j0 + jl;
                pc[q] = pkm[q] = ped[q] = A::zero();
                lc[q] = lkm[q] = led[q] = 0.f;
                ru[q] = rv[q] = rw[q] = rwt[q] = 0.0;
                if (jl < sm.r1 && j < ny) {
                    const int jm = (j == 0) ? ny - 1 : j - 1;
                    const int row = j * nx;
                    if (q == 0 && need0) pjm0 = ph.get(jm * nx + ii);
                    pc[q] = ph.get(row + ii);
                    if (k > 0) pkm[q] = ph.get(row + ii - plane);
                    if (own_dn) ped[q] = ph.get(row + im);
                    if constexpr (L2) {
                        if (q == 0 && need0) ljm0 = __ldg(l2p + jm * nx + ii);
                        lc[q] = __ldg(l2p + row + ii);
                        if (k > 0) lkm[q] = __ldg(l2p + row + ii - plane);
                        if (own_dn) led[q] = __ldg(l2p + row + im);
                    }
                    if (act) {
                        ru[q] = ui[j * nxu + i];
                        rv[q] = vi[row + i];
                        rw[q] = wi[row + i];
                        if (k == nz - 1) rwt[q] = wi[row + i + plane];
                    }
                }
            }
            if (need0) {
                Pjm = pjm0;
                L2jm = ljm0;
            }
            if constexpr (MIX && !ADJ && !PU) {
                // forward, mixed: both rows of the group at once, row jg in the x lane and row
                // jg + 1 in the y lane of packed operations (lane for lane the scalar sequence
                // of the general branch below); the neighbours and the fp64 conversions and
                // stores per row
                static_assert(kRowGroupC == 2, "two rows per packed step");
                bool live[2];
                df Pcs[2], Pims[2], Pjws[2];
                float Lcs[2], dlx[2], dly[2], dlz[2];
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    const int j = j0 + jg + h;
                    live[h] = jg + h < sm.r1 && j < ny;
                    const df Pc = pc[h];
                    df Pim = shup(Pc, 1);
                    if (own_dn) Pim = ped[h];
                    if (wall_lo) Pim = Pc;
                    const df Pjm_h = h == 0 ? Pjm : pc[0];
                    Pcs[h] = Pc;
                    Pims[h] = Pim;
                    Pjws[h] = (wall_y && j == 0) ? Pc : Pjm_h;
                    Lcs[h] = dlx[h] = dly[h] = dlz[h] = 0.f;
                    if constexpr (L2) {
                        const float Lc = lc[h];
                        float Lim = __shfl_up_sync(0xffffffffu, Lc, 1);
                        if (own_dn) Lim = led[h];
                        if (wall_lo) Lim = Lc;
                        const float Ljm_h = h == 0 ? L2jm : lc[0];
                        const float Ljw = (wall_y && j == 0) ? Lc : Ljm_h;
                        Lcs[h] = Lc;
                        dlx[h] = __fsub_rn(Lim, Lc);
                        dly[h] = __fsub_rn(Ljw, Lc);
                        dlz[h] = __fsub_rn(lkm[h], Lc);
                    }
                }
                if (live[0]) {
                    auto pk = [](const df (&v)[2]) {
                        return df2{make_float2(v[0].hi, v[1].hi), make_float2(v[0].lo, v[1].lo)};
                    };
                    auto pkf = [](const float (&v)[2]) { return make_float2(v[0], v[1]); };
                    const df2 P = pk(Pcs);
                    const df2 ZM = {make_float2(pkm[0].hi, pkm[1].hi), make_float2(pkm[0].lo, pkm[1].lo)};
                    auto term2 = [&](df c, df2 d, float2 dl) {  // c d (+ c dl with lo2)
                        df2 t = df_mul2(c, d);
                        if constexpr (L2) {
                            t.lo = __ffma2_rn(make_float2(c.hi, c.hi), dl, t.lo);
                            t = quick_two_sum2(t.hi, t.lo);
                        }
                        return t;
                    };
                    const df2 tx = term2(cu, df_sub2_acc(pk(Pims), P), pkf(dlx));
                    const df2 ty = term2(cv, df_sub2_acc(pk(Pjws), P), pkf(dly));
                    const df2 tz = term2(cw, df_sub2_acc(ZM, P), pkf(dlz));
                    df2 tt = {make_float2(0.f, 0.f), make_float2(0.f, 0.f)};
                    if (k == nz - 1 && G.dir_top) tt = term2(cwt, P, pkf(Lcs));
                    df2 Pn = P;
                    if constexpr (L2) Pn.lo = p2add(P.lo, pkf(Lcs));
                    Pn = quick_two_sum2(Pn.hi, Pn.lo);
#pragma unroll
                    for (int h = 0; h < 2; ++h) {
                        if (!live[h] || !act) continue;
                        const int j = j0 + jg + h, c = j * nx + i;
                        auto lane_of = [h](const df2 &v) {
                            return h == 0 ? df{v.hi.x, v.lo.x} : df{v.hi.y, v.lo.y};
                        };
                        uo[j * nxu + i] = ru[h] + df_to_f64(lane_of(tx));
                        vo[c] = rv[h] + df_to_f64(lane_of(ty));
                        if (k == 0) wo[c] = rw[h];
                        else wo[c] = rw[h] + df_to_f64(lane_of(tz));
                        if (k == nz - 1)  // outlet face: corrected with a Dirichlet outlet, else a wall
                            wo[c + plane] = G.dir_top ? rwt[h] + df_to_f64(lane_of(tt)) : rwt[h];
                        if (po) po[c] = df_to_f64(lane_of(Pn));
                    }
                    Pjm = live[1] ? Pcs[1] : Pcs[0];
                    L2jm = live[1] ? Lcs[1] : Lcs[0];
                    have = true;
                }
            } else {
#pragma unroll
            for (int q = 0; q < kRowGroupC; ++q) {
                const int jl = jg + q, j = j0 + jl;
                if (jl >= sm.r1 || j >= ny) break;  // warp-uniform
                const int row = j * nx;
                const V Pc = pc[q];
                V Pim = shup(Pc, 1);
                if (own_dn) Pim = ped[q];
                // wall faces: no gradient (forward: velocity copied); the adjoint's D^T
                // there sees only the one interior cell
                if (wall_lo) Pim = ADJ ? A::zero() : Pc;
                const V Pjw = (wall_y && j == 0) ? (ADJ ? A::zero() : Pc) : Pjm;
                // L2: the differences of lo2 in fp32 (lo2 is a few 1e-10 of phi), added to
                // the low word of each correction term, which is then renormalised
                float dlx = 0.f, dly = 0.f, dlz = 0.f, Lc = 0.f;
                if constexpr (L2) {
                    Lc = lc[q];
                    float Lim = __shfl_up_sync(0xffffffffu, Lc, 1);
                    if (own_dn) Lim = led[q];
                    if (wall_lo) Lim = ADJ ? 0.f : Lc;
                    const float Ljw = (wall_y && j == 0) ? (ADJ ? 0.f : Lc) : L2jm;
                    dlx = __fsub_rn(Lim, Lc);
                    dly = __fsub_rn(Ljw, Lc);
                    dlz = __fsub_rn(lkm[q], Lc);
                    L2jm = Lc;
                }
                auto term = [&](V c, V d, float dl) {  // c d (+ c dl with lo2), as an fp64 number
                    V t = A::mul(c, d);
                    if constexpr (L2) {
                        t.lo = __fmaf_rn(c.hi, dl, t.lo);
                        t = quick_two_sum(t.hi, t.lo);
                    }
                    return A::store(t);
                };
                auto phi_out = [&](V P) {  // phi (L2: hi + lo + lo2, rounded once) as an fp64 number
                    if constexpr (L2) P.lo = __fadd_rn(P.lo, Lc);
                    return A::store(A::norm(P));
                };
                if (act) {
                    // the correction t is formed in the solve's high precision; the face
                    // value u* + t is one fp64 add (the fp64 pipe is otherwise idle here)
                    const int c = row + i;
                    uo[j * nxu + i] = ru[q] + term(cu, A::sub_acc(Pim, Pc), dlx);
                    vo[c] = rv[q] + term(cv, A::sub_acc(Pjw, Pc), dly);
                    if (ADJ) {
                        wo[c] = rw[q] + term(A::from_f(1.f), A::sub_acc(pkm[q], Pc), dlz);
                        if (k == nz - 1) wo[c + plane] = rwt[q] + phi_out(Pc);
                    } else {
                        if (k == 0) wo[c] = rw[q];
                        else wo[c] = rw[q] + term(cw, A::sub_acc(pkm[q], Pc), dlz);
                        if (k == nz - 1)  // outlet face: corrected with a Dirichlet outlet, else a wall
                            wo[c + plane] = G.dir_top ? rwt[q] + term(cwt, Pc, Lc) : rwt[q];
                        if (po) {
                            if constexpr (!PU) {
                                po[c] = phi_out(Pc);
                            } else {
                                double pv = pn[c] + phi_out(Pc);
                                if (pmode == 2) {
                                    double bb;
                                    if constexpr (MIX) {
                                        const float2 bd = w.bdf[G.cell_off + pbase + c];
                                        bb = df_to_f64(df_sub(df{bd.x, bd.y}, Coef<A>::c(mean_b)));
                                    } else {
                                        bb = w.bws[G.cell_off + pbase + c] - mean_b;
                                    }
                                    pv -= cimp * bb;
                                }
                                po[c] = pv;
                            }
                        }
                    }
                }
                Pjm = Pc;
                have = true;
            }
            }
        }
    }
    // the far wall faces: u face nx of every row (wall-bounded x), v row ny (wall-bounded y)
    if (wall_x) {
        const int nr = min(rows, ny - j0);
        for (int t = threadIdx.x; t < nr; t += blockDim.x) {
            const int j = j0 + t, f = j * nxu + nx;
            V pf = ph.get(j * nx + nx - 1);
            if constexpr (L2) pf = df_addf(pf, __ldg(l2p + j * nx + nx - 1));
            uo[f] = ADJ ? ui[f] + A::store(A::mul(cu, pf)) : ui[f];
        }
    }
    if (wall_y && j0 + rows >= ny) {
        for (int i = threadIdx.x; i < nx; i += blockDim.x) {
            const int f = ny * nx + i;
            V pf = ph.get((ny - 1) * nx + i);
            if constexpr (L2) pf = df_addf(pf, __ldg(l2p + (ny - 1) * nx + i));
            vo[f] = ADJ ? vi[f] + A::store(A::mul(cv, pf)) : vi[f];
        }
    }
}

// ================================================================ k_divstat: max |D u| of the output
template <class A, bool W>
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
    const int wall_x = W ? G.wall_x : 0, wall_y = W ? G.wall_y : 0, nxu = W ? G.nxu : nx;
    const double *u = p.out_u[gi] + (ptrdiff_t)k * ny * nxu, *vv = p.out_v[gi] + (ptrdiff_t)k * (W ? G.nyv : ny) * nx,
                 *ww = p.out_w[gi] + pbase;
    const V cu = Coef<A>::c(G.rdx), cv = Coef<A>::c(G.rdy), cw = Coef<A>::c(w.z.rhz[G.z_off + k]);
    const double *qs = p.in_q[gi] ? p.in_q[gi] + pbase : nullptr;
    float mx = 0.f;
    const int ncell = min(rows, ny - j0) * nx;
    for (int t = threadIdx.x; t < ncell; t += blockDim.x) {
        const int jl = (int)fdiv((unsigned)t, G.fnx), i = t - jl * nx;
        const int j = j0 + jl;
        const int ip = (i + 1 == nx && !wall_x) ? 0 : i + 1;
        const int jp = (j + 1 == ny && !wall_y) ? 0 : j + 1;
        const int row = j * nx, rowu = j * nxu;
        V d = A::mul(cu, A::sub(A::load(u[rowu + ip]), A::load(u[rowu + i])));
        d = A::add(d, A::mul(cv, A::sub(A::load(vv[jp * nx + i]), A::load(vv[row + i]))));
        d = A::add(d, A::mul(cw, A::sub(A::load(ww[plane + row + i]), A::load(ww[row + i]))));
        if (qs) d = A::sub(d, A::load(qs[row + i]));  // constraint D u = q
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


// ================================================================ launchers

template <bool W, int SPLIT>
cudaError_t launch_xfwd_mixed(int mode, const Work &w, const UserPtrs &p, int use_ws, int lo_valid, int nblk,
                              double s, double rs, size_t smem, cudaStream_t st) {
    const dim3 gr = grid1(SPLIT * nblk);
    const int nt = kXThreads / SPLIT;
    smem /= SPLIT;
    if (mode == XM_DIV)
        k_xfwd<float, DFArith, XM_DIV, W, SPLIT><<<gr, nt, smem, st>>>(w, p, use_ws, lo_valid, s, rs);
    else if (mode == XM_DIVQ)
        k_xfwd<float, DFArith, XM_DIVQ, W, SPLIT><<<gr, nt, smem, st>>>(w, p, use_ws, lo_valid, s, rs);
    else if (mode == XM_RESID && !lo_valid)
        k_xfwd<float, DFArith, XM_RESID0, W, SPLIT><<<gr, nt, smem, st>>>(w, p, use_ws, lo_valid, s, rs);
    else if (mode == XM_RESID)
        k_xfwd<float, DFArith, XM_RESID, W, SPLIT><<<gr, nt, smem, st>>>(w, p, use_ws, lo_valid, s, rs);
    else if (mode == XM_RESID1) {
        if (!w.rdf) return cudaErrorInvalidValue;  // the first sweep's residual is not kept
        k_xfwd<float, DFArith, XM_RESID1, W, SPLIT><<<gr, nt, smem, st>>>(w, p, use_ws, lo_valid, s, rs);
    } else if (mode == XM_COPY) {
        if constexpr (W) return cudaErrorInvalidValue;  // periodic x and y only
        else k_xfwd<float, DFArith, XM_COPY, false, SPLIT><<<gr, nt, smem, st>>>(w, p, use_ws, lo_valid, s, rs);
    } else
        k_xfwd<float, DFArith, XM_ADJ, W, SPLIT><<<gr, nt, smem, st>>>(w, p, use_ws, lo_valid, s, rs);
    return cudaGetLastError();
}

template <bool W>
cudaError_t launch_xfwd_w(int mixed, int mode, const Work &w, const UserPtrs &p, int use_ws, int lo_valid, int nblk,
                          double s, double rs, size_t smem, cudaStream_t st) {
    if (mixed)
        return w.xfwd_split ? launch_xfwd_mixed<W, 2>(mode, w, p, use_ws, lo_valid, nblk, s, rs, smem, st)
                            : launch_xfwd_mixed<W, 1>(mode, w, p, use_ws, lo_valid, nblk, s, rs, smem, st);
    if (mode == XM_DIV)
        k_xfwd<double, F64Arith, XM_DIV, W, 1><<<grid1(nblk), kXThreads, smem, st>>>(w, p, use_ws, lo_valid, s, rs);
    else if (mode == XM_DIVQ)
        k_xfwd<double, F64Arith, XM_DIVQ, W, 1><<<grid1(nblk), kXThreads, smem, st>>>(w, p, use_ws, lo_valid, s, rs);
    else if (mode == XM_ADJ)
        k_xfwd<double, F64Arith, XM_ADJ, W, 1><<<grid1(nblk), kXThreads, smem, st>>>(w, p, use_ws, lo_valid, s, rs);
    else if (mode == XM_COPY) {
        if constexpr (W) return cudaErrorInvalidValue;
        else k_xfwd<double, F64Arith, XM_COPY, false, 1><<<grid1(nblk), kXThreads, smem, st>>>(w, p, use_ws, lo_valid, s, rs);
    } else
        return cudaErrorInvalidValue;
    return cudaGetLastError();
}

cudaError_t launch_xfwd(int mixed, int mode, const Work &w, const UserPtrs &p, int use_ws, int lo_valid, int nblk,
                        double s, double rs, size_t smem, cudaStream_t st) {
    if (nblk <= 0) return cudaSuccess;
    return w.walls ? launch_xfwd_w<true>(mixed, mode, w, p, use_ws, lo_valid, nblk, s, rs, smem, st)
                   : launch_xfwd_w<false>(mixed, mode, w, p, use_ws, lo_valid, nblk, s, rs, smem, st);
}

template <bool W>
cudaError_t launch_xinv_w(int mixed, int mode, const Work &w, const UserPtrs &p, int use_ws, int lo_valid, int nblk,
                          size_t smem, cudaStream_t st) {
    if (mixed && w.xinv_split) {
        const dim3 gr = grid1(2 * nblk);
        if (mode == IM_STORE)
            k_xinv<float, DFArith, IM_STORE, W, 2><<<gr, kXThreads / 2, smem / 2, st>>>(w, p, use_ws, lo_valid);
        else if (mode == IM_LAST)
            k_xinv<float, DFArith, IM_LAST, W, 2><<<gr, kXThreads / 2, smem / 2, st>>>(w, p, use_ws, lo_valid);
        else
            k_xinv<float, DFArith, IM_ACCUM, W, 2><<<gr, kXThreads / 2, smem / 2, st>>>(w, p, use_ws, lo_valid);
    } else if (mixed) {
        if (mode == IM_STORE)
            k_xinv<float, DFArith, IM_STORE, W, 1><<<grid1(nblk), kXThreads, smem, st>>>(w, p, use_ws, lo_valid);
        else if (mode == IM_LAST)
            k_xinv<float, DFArith, IM_LAST, W, 1><<<grid1(nblk), kXThreads, smem, st>>>(w, p, use_ws, lo_valid);
        else
            k_xinv<float, DFArith, IM_ACCUM, W, 1><<<grid1(nblk), kXThreads, smem, st>>>(w, p, use_ws, lo_valid);
    } else {
        k_xinv<double, F64Arith, IM_STORE, W, 1><<<grid1(nblk), kXThreads, smem, st>>>(w, p, use_ws, lo_valid);
    }
    return cudaGetLastError();
}

cudaError_t launch_xinv(int mixed, int mode, const Work &w, const UserPtrs &p, int use_ws, int lo_valid, int nblk,
                        size_t smem, cudaStream_t st) {
    if (nblk <= 0) return cudaSuccess;
    return w.walls ? launch_xinv_w<true>(mixed, mode, w, p, use_ws, lo_valid, nblk, smem, st)
                   : launch_xinv_w<false>(mixed, mode, w, p, use_ws, lo_valid, nblk, smem, st);
}

template <bool W>
cudaError_t launch_correct_w(int mixed, int adjoint, const Work &w, const UserPtrs &p, int use_ws, int lo_valid,
                             int lo2, int nblk, double s, int pm, double ci, cudaStream_t st) {
    const dim3 gr = grid1(nblk);
    if (mixed && lo2) {
        if (adjoint) k_correct<DFArith, 1, W, false, true><<<gr, kXThreads, 0, st>>>(w, p, use_ws, lo_valid, s, 0, 0.0);
        else if (pm) k_correct<DFArith, 0, W, true, true><<<gr, kXThreads, 0, st>>>(w, p, use_ws, lo_valid, s, pm, ci);
        else k_correct<DFArith, 0, W, false, true><<<gr, kXThreads, 0, st>>>(w, p, use_ws, lo_valid, s, 0, 0.0);
    } else if (mixed) {
        if (adjoint) k_correct<DFArith, 1, W, false><<<gr, kXThreads, 0, st>>>(w, p, use_ws, lo_valid, s, 0, 0.0);
        else if (pm) k_correct<DFArith, 0, W, true><<<gr, kXThreads, 0, st>>>(w, p, use_ws, lo_valid, s, pm, ci);
        else k_correct<DFArith, 0, W, false><<<gr, kXThreads, 0, st>>>(w, p, use_ws, lo_valid, s, 0, 0.0);
    } else {
        if (adjoint) k_correct<F64Arith, 1, W, false><<<gr, kXThreads, 0, st>>>(w, p, use_ws, lo_valid, s, 0, 0.0);
        else if (pm) k_correct<F64Arith, 0, W, true><<<gr, kXThreads, 0, st>>>(w, p, use_ws, lo_valid, s, pm, ci);
        else k_correct<F64Arith, 0, W, false><<<gr, kXThreads, 0, st>>>(w, p, use_ws, lo_valid, s, 0, 0.0);
    }
    return cudaGetLastError();
}

cudaError_t launch_correct(int mixed, int adjoint, const Work &w, const UserPtrs &p, int use_ws, int lo_valid,
                           int lo2, int nblk, double s, int pmode, double cimp, cudaStream_t st) {
    if (nblk <= 0) return cudaSuccess;
    return w.walls ? launch_correct_w<true>(mixed, adjoint, w, p, use_ws, lo_valid, lo2, nblk, s, pmode, cimp, st)
                   : launch_correct_w<false>(mixed, adjoint, w, p, use_ws, lo_valid, lo2, nblk, s, pmode, cimp, st);
}

cudaError_t launch_divstat(int mixed, const Work &w, const UserPtrs &p, int nblk, cudaStream_t st) {
    if (nblk <= 0) return cudaSuccess;
    if (mixed) {
        if (w.walls) k_divstat<DFArith, true><<<grid1(nblk), kXThreads, 0, st>>>(w, p);
        else k_divstat<DFArith, false><<<grid1(nblk), kXThreads, 0, st>>>(w, p);
    } else {
        if (w.walls) k_divstat<F64Arith, true><<<grid1(nblk), kXThreads, 0, st>>>(w, p);
        else k_divstat<F64Arith, false><<<grid1(nblk), kXThreads, 0, st>>>(w, p);
    }
    return cudaGetLastError();
}

cudaError_t launch_finalize(const Work &w, double *max_div, double *max_div_in, double *compat, double s,
                            cudaStream_t st) {
    k_finalize<<<(w.ngrids + 127) / 128, 128, 0, st>>>(w, max_div, max_div_in, compat, s);
    return cudaGetLastError();
}

// Dynamic shared-memory caps are per-kernel attributes shared by every plan in the
// process: each is set to the device's opt-in maximum minus the kernel's static shared
// memory, so that no plan can lower them under another plan's launch size.
cudaError_t set_smem_cap(const void *fn) {
    int dev = 0, optin = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    cudaFuncAttributes a;
    if (e == cudaSuccess) e = cudaFuncGetAttributes(&a, fn);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, optin - (int)a.sharedSizeBytes);
    return e;
}

cudaError_t set_smem_limits(int mixed) {
    cudaError_t e = cudaSuccess;
    auto set = [&](const void *fn) {
        if (e == cudaSuccess) e = set_smem_cap(fn);
    };
    auto set_all = [&](auto wtag) {
        constexpr bool W = decltype(wtag)::value;
        if (mixed) {
            set((const void *)k_xfwd<float, DFArith, XM_DIV, W, 1>);
            set((const void *)k_xfwd<float, DFArith, XM_DIVQ, W, 1>);
            set((const void *)k_xfwd<float, DFArith, XM_RESID, W, 1>);
            set((const void *)k_xfwd<float, DFArith, XM_RESID0, W, 1>);
            set((const void *)k_xfwd<float, DFArith, XM_RESID1, W, 1>);
            set((const void *)k_xfwd<float, DFArith, XM_ADJ, W, 1>);
            set((const void *)k_xfwd<float, DFArith, XM_DIV, W, 2>);
            set((const void *)k_xfwd<float, DFArith, XM_DIVQ, W, 2>);
            set((const void *)k_xfwd<float, DFArith, XM_RESID, W, 2>);
            set((const void *)k_xfwd<float, DFArith, XM_RESID0, W, 2>);
            set((const void *)k_xfwd<float, DFArith, XM_RESID1, W, 2>);
            set((const void *)k_xfwd<float, DFArith, XM_ADJ, W, 2>);
            set((const void *)k_xinv<float, DFArith, IM_STORE, W, 1>);
            set((const void *)k_xinv<float, DFArith, IM_ACCUM, W, 1>);
            set((const void *)k_xinv<float, DFArith, IM_LAST, W, 1>);
            set((const void *)k_xinv<float, DFArith, IM_STORE, W, 2>);
            set((const void *)k_xinv<float, DFArith, IM_ACCUM, W, 2>);
            set((const void *)k_xinv<float, DFArith, IM_LAST, W, 2>);
        } else {
            set((const void *)k_xfwd<double, F64Arith, XM_DIV, W, 1>);
            set((const void *)k_xfwd<double, F64Arith, XM_DIVQ, W, 1>);
            set((const void *)k_xfwd<double, F64Arith, XM_ADJ, W, 1>);
            set((const void *)k_xinv<double, F64Arith, IM_STORE, W, 1>);
        }
    };
    set_all(std::false_type{});
    set_all(std::true_type{});
    if (mixed) {
        set((const void *)k_xfwd<float, DFArith, XM_COPY, false, 1>);
        set((const void *)k_xfwd<float, DFArith, XM_COPY, false, 2>);
    } else {
        set((const void *)k_xfwd<double, F64Arith, XM_COPY, false, 1>);
    }
    if (e == cudaSuccess) e = set_smem_limits_yz(mixed);
    return e;
}

}  // namespace ibf

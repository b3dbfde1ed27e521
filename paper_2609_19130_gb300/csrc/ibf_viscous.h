// ibf_viscous.h -- launchers of the factored implicit viscous solve (ibf_viscous.cu),
// called by ibf_capi.cpp.  Not part of the public ABI.
#pragma once
#include "ibf_internal.h"

namespace ibf {

constexpr int kZHelmThreads = 256;  // z-Thomas kernel: one thread per (i, j) column

// pivots of (I - beta Lz) for every grid (tab / tabf: 6 (nz+1) entries per grid at 6 z_off)
// and the x / y factors 1/(1 + beta (4/h^2) sin^2(pi m/n)) (fxy / fxyf: nxh + ny entries per
// grid at fxy_off[g], a device array)
cudaError_t launch_helm_table(const Work &w, int ngrids, double beta, double *tab, float *tabf,
                              const long long *fxy_off, double *fxy, float *fxyf, cudaStream_t st);
// y-FFT, x/y factors, inverse y-FFT of grid g: groups of gb column blocks (nblk = nz *
// ceil(ncb / gb) blocks, shared memory for gb mb sequences); fxy / fxyf: grid g's factors
cudaError_t launch_yhelm(int mixed, const Work &w, int g, int nblk, int gb, const double *fxy, const float *fxyf,
                         size_t smem, cudaStream_t st);
// column blocks per k_yhelm CTA: enough sequences (gb mb >= 4) for the FFT passes to reach
// every warp when the blocks are one or two x-modes wide
inline int yhelm_group(int mb) { return mb >= 4 ? 1 : 4 / mb; }
// z-Thomas of grid g's ncol = nx ny columns; zshift 1 for w (interior faces), 0 for u, v
cudaError_t launch_zhelm(int mixed, const Work &w, int g, long long ncol, int zshift, const double *tab,
                         const float *tabf, double *out, cudaStream_t st);
cudaError_t set_smem_limits_visc(int mixed);

}  // namespace ibf

"""Write tests/golden/fullsize_1024x1024x512_oracle.txt: the FP64 oracle's projection of the
1024x1024x512 workload (2 pi x 2 pi x [0, 2], tanh clustering 2.5, k^-5/3 Fourier-mode velocity
of seed 4 plus U[-0.01, 0.01] noise, dt = 1e-3, alpha = 1), reduced to what a test can compare:

  * the oracle's statistics: max|D u| of its output, max|D u*|, the removed compatibility mean;
  * the plane sums sum_ij phi_k of every level k (they carry the (0,0) mode of the solve);
  * phi, u, v and w at sampled cells: 512 drawn over the whole grid and 128 in each of the
    planes 0, 1, nz-2, nz-1 next to the walls (w at the cell's lower face k).

Only the oracle and the seeded input generator run here (the velocity is synthesised on the
host with torch's CPU FFT).  The run needs about 50 GB of host memory and, on 8 cores, about
half an hour:  python tests/golden/make_fullsize_golden.py
"""
import math
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

from oracle import oracle as O  # noqa: E402
from paper_2609_19130_gb300 import synth  # noqa: E402

NX, NY, NZ, BETA, SEED, DT, ALPHA = 1024, 1024, 512, 2.5, 4, 1e-3, 1.0
OUT = os.path.join(HERE, "fullsize_1024x1024x512_oracle.txt")
SAMPLE_SEED = 4104  # splitmix64 seed of the sample positions


def sample_positions(nx, ny, nz):
    """(k, j, i) of the sampled cells: 512 over the grid, 128 in each near-wall plane."""
    def draw(aid, n, mod):
        return (synth.bits_np(SAMPLE_SEED, aid, n) % np.uint64(mod)).astype(np.int64)
    pos = list(zip(draw(1, 512, nz), draw(2, 512, ny), draw(3, 512, nx)))
    for t, k in enumerate((0, 1, nz - 2, nz - 1)):
        pos += [(k, j, i) for j, i in zip(draw(10 + t, 128, ny), draw(20 + t, 128, nx))]
    return pos


def main():
    import torch
    t0 = time.time()
    u, v, w = (t.numpy() for t in synth.kolmogorov_velocity_torch(SEED, NX, NY, NZ, "cpu"))
    print(f"inputs {time.time() - t0:.0f} s", flush=True)
    g = O.Grid(NX, NY, NZ, lx=2 * math.pi, ly=2 * math.pi, lz=2.0, beta=BETA)
    phi, uo, vo, wo, st = O.project(g, u, v, w, dt=DT, alpha=ALPHA)
    print(f"oracle {time.time() - t0:.0f} s: stats {st}", flush=True)
    psum = phi.reshape(NZ, -1).sum(axis=1)
    with open(OUT, "w") as f:
        f.write("# FP64 oracle (oracle/ibf_oracle.c) projection of the 1024x1024x512 workload, written by\n")
        f.write("# tests/golden/make_fullsize_golden.py: lx = ly = 2 pi, lz = 2, tanh clustering 2.5,\n")
        f.write("# synth.kolmogorov_velocity_torch(seed 4) on the host, dt = 1e-3, alpha = 1.\n")
        f.write(f"grid {NX} {NY} {NZ} {BETA!r} {SEED} {DT!r} {ALPHA!r}\n")
        r = lambda x: repr(float(x))
        f.write(f"stats {r(st[0])} {r(st[1])} {r(st[2])}\n")
        f.write(f"umax {r(max(np.abs(u).max(), np.abs(v).max(), np.abs(w).max()))}\n")
        f.write(f"phimax {r(np.abs(phi).max())}\n")
        f.write(f"phinorm {r(np.linalg.norm(phi))}\n")
        f.write("# plane k, sum over the plane of phi_k\n")
        for k in range(NZ):
            f.write(f"psum {k} {r(psum[k])}\n")
        f.write("# k j i phi u v w (w at the lower face k of the cell)\n")
        for k, j, i in sample_positions(NX, NY, NZ):
            f.write(f"s {k} {j} {i} {r(phi[k, j, i])} {r(uo[k, j, i])} {r(vo[k, j, i])} {r(wo[k, j, i])}\n")
    print(f"wrote {OUT} ({time.time() - t0:.0f} s)")


if __name__ == "__main__":
    main()

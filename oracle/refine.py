"""Extended-precision refinement of the oracle's Poisson solve.  Test infrastructure only.

On a strongly stretched z (the benchmark's tanh clustering 2.5 with 512 levels: faces
2.7e-4 apart at the walls, 2 / 512 on average) the tridiagonal systems of the low
horizontal modes are ill-conditioned, and the oracle's plain FP64 solve (naive DFT +
Thomas, oracle/ibf_oracle.c) carries a forward error of a few 1e-12 of phi: more than
the 1e-12 that parity asks of the FP64 path.  This module gives the exact discrete
solution to beyond FP64 accuracy by iterative refinement (Wilkinson), the oracle's own
solve applied to residuals evaluated in extended precision:

    phi_0 = S(b),   r_s = (b - <b>_V) - L phi_s   (numpy longdouble),
    phi_{s+1} = phi_s + S(r_s)                    (S: oracle.poisson, FP64).

L is the discrete Laplacian of the projection (Section "Fluid Mechanics", Eq.
(elliptic); staggered second-order differences, periodic x and y, Neumann walls in z
or a homogeneous Dirichlet outlet on top), written out here from its definition in
longdouble; the weighted-mean conventions of phi are those of the oracle (the
reference value of phi, same section, boundary-condition paragraph).  Only periodic x
and y are supported.  Nothing here is imported by the product.
"""
from __future__ import annotations

import numpy as np

from . import oracle as O

LD = np.longdouble


def _metrics(g: O.Grid):
    zf = np.asarray(g.zf, dtype=LD)
    hz = zf[1:] - zf[:-1]
    zc = LD(0.5) * (zf[1:] + zf[:-1])
    rg = np.zeros(g.nz + 1, dtype=LD)          # 1 / gz on the interior faces, 0 on walls
    rg[1:g.nz] = LD(1) / (zc[1:] - zc[:-1])
    if g.dirichlet_top:                         # outlet face: phi = 0 on it
        rg[g.nz] = LD(1) / (zf[g.nz] - zc[g.nz - 1])
    return hz, rg


def laplacian_ld(g: O.Grid, phi) -> np.ndarray:
    """L phi in longdouble: x and y second differences (periodic) plus the z flux
    differences (F_k - F_{k-1}) / hz_k with F on the faces, zero on Neumann walls."""
    if g.wall_x or g.wall_y:
        raise ValueError("periodic x and y only")
    p = np.asarray(phi, dtype=LD)
    dx, dy = LD(g.lx) / g.nx, LD(g.ly) / g.ny
    hz, rg = _metrics(g)
    r = (np.roll(p, -1, 2) - 2 * p + np.roll(p, 1, 2)) / (dx * dx)
    r += (np.roll(p, -1, 1) - 2 * p + np.roll(p, 1, 1)) / (dy * dy)
    F = np.zeros((g.nz + 1, g.ny, g.nx), dtype=LD)
    F[1:g.nz] = (p[1:] - p[:-1]) * rg[1:g.nz, None, None]
    if g.dirichlet_top:
        F[g.nz] = (LD(0) - p[-1]) * rg[g.nz]
    return r + (F[1:] - F[:-1]) / hz[:, None, None]


def _weighted_mean(g: O.Grid, a) -> LD:
    hz, _ = _metrics(g)
    return (hz[:, None, None] * np.asarray(a, dtype=LD)).sum() / (hz.sum() * g.nx * g.ny)


def refined_poisson(g: O.Grid, b, sweeps: int = 2):
    """The exact discrete solution of L phi = b - <b>_V with <phi>_V = 0 (or, with a
    Dirichlet outlet, of L phi = b), to beyond FP64 accuracy: the oracle's solve, then
    `sweeps` corrections from longdouble residuals.  b may be float64 or longdouble.
    Returns (phi as float64, max|residual| of each step)."""
    bl = np.asarray(b, dtype=LD)
    if not g.dirichlet_top:
        bl = bl - _weighted_mean(g, bl)
    phi, _ = O.poisson(g, np.asarray(bl, dtype=np.float64))
    cur = phi.astype(LD)
    res = []
    for _ in range(sweeps):
        r = bl - laplacian_ld(g, cur)
        res.append(float(np.abs(r).max()))
        d, _ = O.poisson(g, np.asarray(r, dtype=np.float64))
        cur = cur + d.astype(LD)
    if not g.dirichlet_top:
        cur = cur - _weighted_mean(g, cur)
    return np.asarray(cur, dtype=np.float64), res


def refined_project(g: O.Grid, us, vs, ws, dt=1e-3, alpha=1.0, sweeps: int = 2):
    """phi of the projection (Eq. elliptic with q = 0) refined as above; returns phi."""
    b = O.divergence(g, us, vs, ws) / (alpha * dt)
    phi, _ = refined_poisson(g, b, sweeps)
    return phi

"""FP64 oracle of the factored implicit viscous solve.  TEST INFRASTRUCTURE ONLY:
only tests/, __graft_entry__.smoke() and bench.py's CPU leg import it; the CUDA
library never does, and nothing here comes from it.

Section "Fluid Mechanics", Eq. (nstime_discr): with the viscous terms advanced by
Crank-Nicolson the provisional velocity carries (alpha / 2 Re) lap(u_hat + u_n).
Section "Fluid domain" (provisional-step paragraph) states how the paper solves
it: the implicit operator is split into one tridiagonal solve per direction,
Thomas' algorithm, with a Sherman-Morrison perturbation for the two periodic
directions.  For one velocity component the factored solve is

    out = (I - beta Lz)^-1 (I - beta Ly)^-1 (I - beta Lx)^-1 rhs,
    beta = alpha dt / (2 Re),

taken here in the order x, y, z, with the algorithms the paper names: Thomas
with the Sherman-Morrison correction on every periodic x and y line, plain
Thomas on every z line.

Readings where the paper is silent (listed in the design notes as V1-V3):
 V1 x, y periodic and uniform: (Lx f)_i = (f_{i+1} - 2 f_i + f_{i-1}) / dx^2 for
    every component (u lives on x-faces, v on y-faces; both are periodic like
    the cells, with the same spacing).
 V2 z for u and v (cell centres k = 0..nz-1, no-slip walls at zf_0 and zf_nz):
      (Lz f)_k = [(f_{k+1} - f_k)/(zc_{k+1} - zc_k) - (f_k - f_{k-1})/(zc_k - zc_{k-1})] / hz_k,
    the wall value zero imposed by a mirror ghost f_{-1} = -f_0 at distance hz_0
    below the first centre (lower flux 2 f_0 / hz_0), likewise at the top.
 V3 z for w (faces k = 1..nz-1; the wall faces k = 0 and nz stay zero):
      (Lz f)_k = [(f_{k+1} - f_k)/hz_k - (f_k - f_{k-1})/hz_{k-1}] / (zc_k - zc_{k-1}).

Arrays are float64 [k][j][i], i fastest: u, v (nz, ny, nx); w (nz+1, ny, nx).
"""
from __future__ import annotations

import numpy as np


def thomas(sub, diag, sup, d):
    """Thomas' algorithm along the last axis: sub[k] f_{k-1} + diag[k] f_k + sup[k] f_{k+1}
    = d_k, k < n (sub[0], sup[n-1] unused).  Coefficients are 1-D (length n), shared by
    every line; d may have any leading shape."""
    d = np.array(d, dtype=np.float64)
    n = d.shape[-1]
    cp = np.empty(n)
    dp = np.empty_like(d)
    cp[0] = sup[0] / diag[0] if n > 1 else 0.0
    dp[..., 0] = d[..., 0] / diag[0]
    for k in range(1, n):
        den = diag[k] - sub[k] * cp[k - 1]
        cp[k] = sup[k] / den if k < n - 1 else 0.0
        dp[..., k] = (d[..., k] - sub[k] * dp[..., k - 1]) / den
    x = np.empty_like(d)
    x[..., n - 1] = dp[..., n - 1]
    for k in range(n - 2, -1, -1):
        x[..., k] = dp[..., k] - cp[k] * x[..., k + 1]
    return x


def cyclic_thomas(sub, diag, sup, corner_lo, corner_hi, d):
    """Cyclic tridiagonal solve along the last axis, n >= 3: the tridiagonal matrix plus
    A[n-1][0] = corner_lo and A[0][n-1] = corner_hi.  Sherman-Morrison: A = B + u v^T with
    u = (g, 0, .., 0, corner_lo), v = (1, 0, .., 0, corner_hi / g), g = -diag[0]; B is
    tridiagonal with its two corner diagonal entries modified; two Thomas solves
    B y = d, B z = u, then x = y - (v.y / (1 + v.z)) z."""
    n = d.shape[-1]
    g = -diag[0]
    bb = np.array(diag, dtype=np.float64)
    bb[0] = diag[0] - g
    bb[n - 1] = diag[n - 1] - corner_lo * corner_hi / g
    y = thomas(sub, bb, sup, d)
    u = np.zeros(n)
    u[0] = g
    u[n - 1] = corner_lo
    z = thomas(sub, bb, sup, u)
    fact = (y[..., 0] + corner_hi * y[..., n - 1] / g) / (1.0 + z[0] + corner_hi * z[n - 1] / g)
    return y - fact[..., None] * z


def periodic_solve(d, h, beta):
    """(I - beta L)^-1 d along the last axis for the periodic second difference with
    spacing h (reading V1)."""
    n = d.shape[-1]
    s = beta / (h * h)
    if n == 1:  # one periodic point: L f = 0
        return np.array(d, dtype=np.float64)
    if n == 2:  # f_{i+1} = f_{i-1}: (L f)_0 = 2 (f_1 - f_0) / h^2
        a, b = 1.0 + 2.0 * s, -2.0 * s
        det = a * a - b * b
        return np.stack([(a * d[..., 0] - b * d[..., 1]) / det, (a * d[..., 1] - b * d[..., 0]) / det], axis=-1)
    sub = np.full(n, -s)
    sup = np.full(n, -s)
    diag = np.full(n, 1.0 + 2.0 * s)
    return cyclic_thomas(sub, diag, sup, -s, -s, d)


def lz_cell(zf):
    """(sub, diag, sup) of Lz on the cell centres (reading V2)."""
    zf = np.asarray(zf, dtype=np.float64)
    nz = len(zf) - 1
    hz = np.diff(zf)
    zc = 0.5 * (zf[1:] + zf[:-1])
    lo = np.empty(nz)
    up = np.empty(nz)
    for k in range(nz):
        dlo = zc[k] - zc[k - 1] if k > 0 else hz[0]           # to the mirror ghost below
        dup = zc[k + 1] - zc[k] if k < nz - 1 else hz[nz - 1]  # to the mirror ghost above
        lo[k] = 1.0 / (dlo * hz[k])
        up[k] = 1.0 / (dup * hz[k])
    sub, sup, diag = lo.copy(), up.copy(), -(lo + up)
    diag[0] -= lo[0]        # ghost f_{-1} = -f_0
    diag[nz - 1] -= up[nz - 1]  # ghost f_nz = -f_{nz-1}
    sub[0] = 0.0
    sup[nz - 1] = 0.0
    return sub, diag, sup


def lz_face(zf):
    """(sub, diag, sup) of Lz on the interior z-faces k = 1..nz-1 (reading V3), indexed
    0..nz-2."""
    zf = np.asarray(zf, dtype=np.float64)
    nz = len(zf) - 1
    hz = np.diff(zf)
    zc = 0.5 * (zf[1:] + zf[:-1])
    m = nz - 1
    sub, diag, sup = np.zeros(m), np.zeros(m), np.zeros(m)
    for r in range(m):
        k = r + 1
        dzc = zc[k] - zc[k - 1]
        lo = 1.0 / (hz[k - 1] * dzc)
        up = 1.0 / (hz[k] * dzc)
        diag[r] = -(lo + up)
        if r > 0:
            sub[r] = lo
        if r < m - 1:
            sup[r] = up
    return sub, diag, sup


def z_solve(d, lz, beta):
    """(I - beta Lz)^-1 d along the last axis, Lz given as (sub, diag, sup)."""
    sub, diag, sup = lz
    return thomas(-beta * sub, 1.0 - beta * diag, -beta * sup, d)


def viscous_solve(nx, ny, nz, lx, ly, zf, ru, rv, rw, beta):
    """Factored implicit viscous solve of the three velocity components (module
    docstring).  Returns (du, dv, dw); dw[0] and dw[nz] are zero."""
    dx, dy = lx / nx, ly / ny
    out = []
    for comp, r in (("u", ru), ("v", rv), ("w", rw)):
        r = np.asarray(r, dtype=np.float64)
        f = r[1:nz] if comp == "w" else r                 # w: interior faces only
        f = periodic_solve(f, dx, beta)                   # x lines (last axis)
        f = np.moveaxis(periodic_solve(np.moveaxis(f, 1, -1), dy, beta), -1, 1)  # y lines
        lz = lz_face(zf) if comp == "w" else lz_cell(zf)
        if f.shape[0] > 0:
            f = np.moveaxis(z_solve(np.moveaxis(f, 0, -1), lz, beta), -1, 0)        # z lines
        if comp == "w":
            full = np.zeros_like(r)
            full[1:nz] = f
            f = full
        out.append(f)
    return tuple(out)

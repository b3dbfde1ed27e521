"""Dense brute-force checker for the projection (test infrastructure only).

Independent of ibf_oracle.c: the operators are assembled here as sparse
matrices from the face/cell incidence of the staggered grid (reading R1/R2 of
the oracle header), L = D G is formed as a dense matrix, and the weighted
pseudo-inverse is obtained by one dense LU solve of the bordered system

    [ L    1 ] [phi]   [b]
    [ V^T  0 ] [ s ] = [0]

whose solution satisfies L phi = b - <b>_V and <phi>_V = 0 (s = <b>_V).
Meant for a few thousand cells at most.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp


def operators(nx, ny, nz, lx, ly, zf, wall_x=False, wall_y=False, dirichlet_top=False):
    """Return (D, G, Vc) with D: faces -> cells, G: cells -> faces (sparse CSR).

    Face ordering: all u faces, then v faces, then w faces, each [k][j][i].  With a
    Dirichlet outlet, phi = 0 on the top face: G there is the one-sided difference to
    that face, (0 - phi_{nz-1}) / (zf_nz - zc_{nz-1})."""
    zf = np.asarray(zf, dtype=np.float64)
    dx, dy = lx / nx, ly / ny
    hz = zf[1:] - zf[:-1]
    zc = 0.5 * (zf[1:] + zf[:-1])
    nxu = nx + 1 if wall_x else nx
    nyv = ny + 1 if wall_y else ny
    nu, nv, nw = nz * ny * nxu, nz * nyv * nx, (nz + 1) * ny * nx
    nf, ncells = nu + nv + nw, nx * ny * nz

    def cid(k, j, i):
        return (k * ny + j) * nx + i

    def uid(k, j, i):
        return (k * ny + j) * nxu + i

    def vid(k, j, i):
        return nu + (k * nyv + j) * nx + i

    def wid(k, j, i):
        return nu + nv + (k * ny + j) * nx + i

    rows, cols, vals = [], [], []          # D entries (cell row, face col)
    grows, gcols, gvals = [], [], []       # G entries (face row, cell col)
    for k in range(nz):
        for j in range(ny):
            for i in range(nx):
                c = cid(k, j, i)
                # the two x faces of cell c: left face i, right face i+1
                right = i + 1 if wall_x else (i + 1) % nx
                rows += [c, c]; cols += [uid(k, j, right), uid(k, j, i)]; vals += [1 / dx, -1 / dx]
                top = j + 1 if wall_y else (j + 1) % ny
                rows += [c, c]; cols += [vid(k, top, i), vid(k, j, i)]; vals += [1 / dy, -1 / dy]
                rows += [c, c]; cols += [wid(k + 1, j, i), wid(k, j, i)]; vals += [1 / hz[k], -1 / hz[k]]
    # gradient on interior faces only
    for k in range(nz):
        for j in range(ny):
            for i in range(nxu):
                if wall_x and (i == 0 or i == nx):
                    continue
                grows += [uid(k, j, i)] * 2
                gcols += [cid(k, j, i % nx), cid(k, j, (i - 1) % nx)]
                gvals += [1 / dx, -1 / dx]
        for jj in range(nyv):
            if wall_y and (jj == 0 or jj == ny):
                continue
            for i in range(nx):
                grows += [vid(k, jj, i)] * 2
                gcols += [cid(k, jj % ny, i), cid(k, (jj - 1) % ny, i)]
                gvals += [1 / dy, -1 / dy]
    for k in range(1, nz):
        gz = zc[k] - zc[k - 1]
        for j in range(ny):
            for i in range(nx):
                grows += [wid(k, j, i)] * 2
                gcols += [cid(k, j, i), cid(k - 1, j, i)]
                gvals += [1 / gz, -1 / gz]
    if dirichlet_top:
        gtop = zf[nz] - zc[nz - 1]
        for j in range(ny):
            for i in range(nx):
                grows += [wid(nz, j, i)]
                gcols += [cid(nz - 1, j, i)]
                gvals += [-1 / gtop]
    D = sp.csr_matrix((vals, (rows, cols)), shape=(ncells, nf))
    G = sp.csr_matrix((gvals, (grows, gcols)), shape=(nf, ncells))
    Vc = np.repeat(dx * dy * hz, nx * ny)
    return D, G, Vc


class DenseProjection:
    """P(u*) and its exact transpose with dense linear algebra."""

    def __init__(self, nx, ny, nz, lx, ly, zf, wall_x=False, wall_y=False, dirichlet_top=False):
        self.shape = (nx, ny, nz)
        self.wall_x, self.wall_y = wall_x, wall_y
        self.D, self.G, self.Vc = operators(nx, ny, nz, lx, ly, zf, wall_x, wall_y, dirichlet_top)
        n = nx * ny * nz
        L = (self.D @ self.G).toarray()
        if dirichlet_top:                 # nonsingular: no bordering
            A = L
        else:
            A = np.zeros((n + 1, n + 1))
            A[:n, :n] = L
            A[:n, n] = 1.0
            A[n, :n] = self.Vc
        self.A = A
        self.Ainv = np.linalg.inv(A)      # small problems only
        self.n = n
        # S^-1 as an explicit n x n matrix: phi = Sinv b
        self.Sinv = self.Ainv[:n, :n]
        nxu = nx + 1 if wall_x else nx
        nyv = ny + 1 if wall_y else ny
        self.nu, self.nv, self.nw = nz * ny * nxu, nz * nyv * nx, (nz + 1) * ny * nx
        self.fshapes = ((nz, ny, nxu), (nz, nyv, nx), (nz + 1, ny, nx))

    def flat(self, u, v, w):
        return np.concatenate([np.ravel(u), np.ravel(v), np.ravel(w)])

    def unflat(self, f):
        a = f[:self.nu].reshape(self.fshapes[0])
        b = f[self.nu:self.nu + self.nv].reshape(self.fshapes[1])
        c = f[self.nu + self.nv:].reshape(self.fshapes[2])
        return a, b, c

    def solve(self, b):
        rhs = np.ravel(b) if self.A.shape[0] == self.n else np.concatenate([np.ravel(b), [0.0]])
        x = np.linalg.solve(self.A, rhs)
        return x[:self.n]

    def project(self, us, vs, ws, dt=1e-3, alpha=1.0):
        s = alpha * dt
        f = self.flat(us, vs, ws)
        b = self.D @ f / s
        phi = self.Sinv @ b
        u = f - s * (self.G @ phi)
        nx, ny, nz = self.shape
        return phi.reshape(nz, ny, nx), *self.unflat(u)

    def project_T(self, gu, gv, gw, gphi=None, dt=1e-3, alpha=1.0):
        """Exact transpose of u* -> (u, phi): J^T (g_u, g_phi) with dense S^-1 transposed."""
        s = alpha * dt
        g = self.flat(gu, gv, gw)
        # Jacobians: phi = M f, M = Sinv D / s ;  u = f - s G M f
        Dt = self.D.T.toarray()
        Gt = self.G.T.toarray()
        SinvT = self.Sinv.T
        h = -(Gt @ g) * s
        if gphi is not None:
            h = h + np.ravel(gphi)
        out = g + Dt @ (SinvT @ h) / s
        return self.unflat(out)

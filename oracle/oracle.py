"""ctypes front end of the C oracle (FP64).  Test infrastructure only.

Every function mirrors one entry point of ibf_oracle.c; arrays are numpy
float64, C-contiguous, laid out [k][j][i] with i fastest:
  u (nz, ny, nx or nx+1), v (nz, ny or ny+1, nx), w (nz+1, ny, nx), phi (nz, ny, nx).
"""
from __future__ import annotations

import ctypes as C
from dataclasses import dataclass

import numpy as np

from . import build_oracle

_lib = None


def lib():
    global _lib
    if _lib is None:
        _lib = C.CDLL(build_oracle.build())
        dp = C.POINTER(C.c_double)
        _lib.ibfo_zfaces_tanh.argtypes = [C.c_int, C.c_double, C.c_double, dp]
        for name in ("ibfo_divergence",):
            getattr(_lib, name).argtypes = [C.c_void_p, dp, dp, dp, dp]
        _lib.ibfo_gradient.argtypes = [C.c_void_p, dp, dp, dp, dp]
        _lib.ibfo_laplacian.argtypes = [C.c_void_p, dp, dp]
        _lib.ibfo_gradient_T.argtypes = [C.c_void_p, dp, dp, dp, dp]
        _lib.ibfo_divergence_T.argtypes = [C.c_void_p, dp, dp, dp, dp]
        _lib.ibfo_poisson.argtypes = [C.c_void_p, dp, dp, dp]
        _lib.ibfo_project.argtypes = [C.c_void_p, dp, dp, dp, C.c_double, C.c_double, dp, dp, dp, dp, dp]
        _lib.ibfo_project_adjoint.argtypes = [C.c_void_p, dp, dp, dp, dp, C.c_double, C.c_double, dp, dp, dp]
        _lib.ibfo_dft.argtypes = [dp, dp, dp, dp, C.c_int, C.c_int, C.c_int]
    return _lib


class _CGrid(C.Structure):
    _fields_ = [("nx", C.c_int), ("ny", C.c_int), ("nz", C.c_int),
                ("lx", C.c_double), ("ly", C.c_double),
                ("zf", C.POINTER(C.c_double)), ("wall_x", C.c_int), ("wall_y", C.c_int),
                ("dirichlet_top", C.c_int)]


def _p(a):
    return a.ctypes.data_as(C.POINTER(C.c_double))


def zfaces_tanh(nz, lz, beta):
    zf = np.empty(nz + 1)
    lib().ibfo_zfaces_tanh(nz, lz, beta, _p(zf))
    return zf


@dataclass
class Grid:
    nx: int
    ny: int
    nz: int
    lx: float = 1.0
    ly: float = 1.0
    lz: float = 1.0
    beta: float = 0.0
    zf: np.ndarray | None = None
    wall_x: bool = False
    wall_y: bool = False
    dirichlet_top: bool = False

    def __post_init__(self):
        if self.zf is None:
            self.zf = zfaces_tanh(self.nz, self.lz, self.beta)
        self.zf = np.ascontiguousarray(self.zf, dtype=np.float64)
        self._c = _CGrid(self.nx, self.ny, self.nz, self.lx, self.ly, _p(self.zf),
                         int(self.wall_x), int(self.wall_y), int(self.dirichlet_top))

    @property
    def cptr(self):
        return C.byref(self._c)

    @property
    def shapes(self):
        nx, ny, nz = self.nx, self.ny, self.nz
        return ((nz, ny, nx + 1 if self.wall_x else nx), (nz, ny + 1 if self.wall_y else ny, nx),
                (nz + 1, ny, nx))

    @property
    def cshape(self):
        return (self.nz, self.ny, self.nx)

    @property
    def hz(self):
        return np.diff(self.zf)


def _c(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def divergence(g: Grid, u, v, w):
    out = np.empty(g.cshape)
    lib().ibfo_divergence(g.cptr, _p(_c(u)), _p(_c(v)), _p(_c(w)), _p(out))
    return out


def gradient(g: Grid, phi):
    su, sv, sw = g.shapes
    gu, gv, gw = np.empty(su), np.empty(sv), np.empty(sw)
    lib().ibfo_gradient(g.cptr, _p(_c(phi)), _p(gu), _p(gv), _p(gw))
    return gu, gv, gw


def laplacian(g: Grid, phi):
    out = np.empty(g.cshape)
    lib().ibfo_laplacian(g.cptr, _p(_c(phi)), _p(out))
    return out


def gradient_T(g: Grid, gu, gv, gw):
    out = np.empty(g.cshape)
    lib().ibfo_gradient_T(g.cptr, _p(_c(gu)), _p(_c(gv)), _p(_c(gw)), _p(out))
    return out


def divergence_T(g: Grid, c):
    su, sv, sw = g.shapes
    gu, gv, gw = np.empty(su), np.empty(sv), np.empty(sw)
    lib().ibfo_divergence_T(g.cptr, _p(_c(c)), _p(gu), _p(gv), _p(gw))
    return gu, gv, gw


def poisson(g: Grid, b):
    """phi = S^-1 b (weighted-mean conventions); returns (phi, removed mean of b)."""
    phi = np.empty(g.cshape)
    compat = C.c_double(0.0)
    b = _c(b)
    lib().ibfo_poisson(g.cptr, _p(b), _p(phi), C.byref(compat))
    return phi, compat.value


def project(g: Grid, us, vs, ws, dt=1e-3, alpha=1.0):
    """Returns (phi, u, v, w, stats) with stats = [max|Du|, max|Du*|, compat, 0]."""
    su, sv, sw = g.shapes
    phi = np.empty(g.cshape)
    u, v, w = np.empty(su), np.empty(sv), np.empty(sw)
    st = np.zeros(4)
    lib().ibfo_project(g.cptr, _p(_c(us)), _p(_c(vs)), _p(_c(ws)), dt, alpha,
                       _p(phi), _p(u), _p(v), _p(w), _p(st))
    return phi, u, v, w, st


def project_q(g: Grid, us, vs, ws, q, dt=1e-3, alpha=1.0):
    """Eq. (elliptic) with a mass source: lap(phi) = (D u* - q)/(alpha dt), then Eq. (velsolen)
    u = u* - alpha dt G phi.  Returns (phi, u, v, w, removed weighted mean of the rhs)."""
    b = (divergence(g, us, vs, ws) - np.asarray(q, dtype=np.float64)) / (alpha * dt)
    phi, compat = poisson(g, b)
    gu, gv, gw = gradient(g, phi)
    s = alpha * dt
    return phi, us - s * gu, vs - s * gv, ws - s * gw, compat


def pressure_update(g: Grid, p_n, phi, dt=1e-3, alpha=1.0, inv_re=0.0):
    """Eq. (pressure) (Section "Fluid Mechanics"): p_{n+1} = p_n + phi - alpha dt/(2 Re) lap(phi),
    with the discrete Laplacian L = D G of the projection; inv_re = 0 is the explicit-viscous
    update p_n + phi."""
    return p_n + phi - 0.5 * alpha * dt * inv_re * laplacian(g, phi)


def project_adjoint(g: Grid, gu, gv, gw, gphi=None, dt=1e-3, alpha=1.0):
    su, sv, sw = g.shapes
    a, b, c = np.empty(su), np.empty(sv), np.empty(sw)
    gp = _p(_c(gphi)) if gphi is not None else C.cast(None, C.POINTER(C.c_double))
    lib().ibfo_project_adjoint(g.cptr, _p(_c(gu)), _p(_c(gv)), _p(_c(gw)), gp, dt, alpha,
                               _p(a), _p(b), _p(c))
    return a, b, c


def dft(x, inverse=False, dct=False):
    x = np.asarray(x)
    n = x.size
    re = _c(np.real(x))
    im = _c(np.imag(x)) if np.iscomplexobj(x) else np.zeros(n)
    ore, oim = np.empty(n), np.empty(n)
    lib().ibfo_dft(_p(re), _p(im), _p(ore), _p(oim), n, int(inverse), int(dct))
    return ore + 1j * oim

"""Pins of the FP64 oracle against facts fixed by the paper and by mathematics.

Each test checks the oracle against something other than itself: a dense
direct solve assembled independently (oracle/dense.py), closed-form discrete
eigenfunctions, a manufactured solution, the O(h^2) convergence of the scheme,
a 1-D case solved by two cumulative sums, library transforms, invariants of the
projection, and the time-scheme coefficients printed in the paper.
"""
import math
from fractions import Fraction

import numpy as np
import pytest

from oracle import dense
from oracle import oracle as O
from paper_2609_19130_gb300 import synth

TOL = 1e-12


def rel(a, b):
    return float(np.max(np.abs(np.asarray(a) - np.asarray(b))) / max(np.max(np.abs(b)), 1e-300))


def vmean(g, f):
    V = g.hz[:, None, None] * np.ones((1, g.ny, g.nx))
    return float(np.sum(V * f) / np.sum(V))


# ---------------------------------------------------------------- dense brute force
@pytest.mark.parametrize("shape,beta,walls", [
    ((8, 8, 8), 0.0, (False, False)),
    ((8, 8, 8), 2.0, (False, False)),
    ((6, 12, 8), 2.0, (False, False)),     # radix-3 sizes
    ((8, 8, 16), 2.5, (False, False)),
    ((8, 6, 5), 1.5, (True, False)),       # wall-bounded x (DCT)
    ((6, 8, 4), 1.5, (False, True)),       # wall-bounded y (DCT)
    ((1, 1, 12), 2.0, (False, False)),     # 1-D column
])
def test_projection_matches_dense_solve(shape, beta, walls):
    nx, ny, nz = shape
    g = O.Grid(nx, ny, nz, lx=1.3, ly=0.7, lz=2.0, beta=beta, wall_x=walls[0], wall_y=walls[1])
    u, v, w = synth.uniform_velocity_np(0, nx, ny, nz, *walls)
    phi, uu, vv, ww, st = O.project(g, u, v, w, dt=1e-3, alpha=1.0)
    dp = dense.DenseProjection(nx, ny, nz, 1.3, 0.7, g.zf, *walls)
    phid, ud, vd, wd = dp.project(u, v, w, dt=1e-3, alpha=1.0)
    assert rel(phi, phid) < TOL
    for a, b in ((uu, ud), (vv, vd), (ww, wd)):
        assert np.max(np.abs(a - b)) < TOL * max(1.0, np.max(np.abs(b)))


def test_incompatible_rhs_dense():
    """Wall fluxes that do not cancel: both remove the same weighted mean of b."""
    nx, ny, nz = 6, 6, 6
    g = O.Grid(nx, ny, nz, lx=1.0, ly=1.0, lz=1.0, beta=1.2)
    u, v, w = synth.uniform_velocity_np(3, nx, ny, nz, zero_walls=False)
    phi, uu, vv, ww, st = O.project(g, u, v, w)
    dp = dense.DenseProjection(nx, ny, nz, 1.0, 1.0, g.zf)
    phid, *_ = dp.project(u, v, w)
    assert rel(phi, phid) < TOL
    assert abs(st[2]) > 1e-3          # a real compatibility defect was removed


# ---------------------------------------------------------------- closed forms
def _eig_lambda(m, n, h, dct):
    s = math.sin(math.pi * m / (2 * n)) if dct else math.sin(math.pi * m / n)
    return -4.0 / h ** 2 * s * s


@pytest.mark.parametrize("a,b,c,walls", [
    (1, 0, 0, (False, False)), (0, 2, 0, (False, False)), (0, 0, 3, (False, False)),
    (3, 5, 2, (False, False)), (7, 1, 5, (False, False)), (2, 3, 1, (True, False)),
    (1, 2, 4, (False, True)), (5, 5, 5, (True, True)),
])
def test_discrete_eigenfunctions(a, b, c, walls):
    """On uniform z, cos-products are eigenfunctions of L = D G with the textbook
    eigenvalues of the second difference (periodic: 4/h^2 sin^2(pi m/N); Neumann
    cell-centred: 4/h^2 sin^2(pi m/2N)); the solver must return them exactly."""
    nx, ny, nz = 16, 12, 10
    lx, ly, lz = 1.7, 0.9, 1.3
    g = O.Grid(nx, ny, nz, lx=lx, ly=ly, lz=lz, beta=0.0, wall_x=walls[0], wall_y=walls[1])
    i = np.arange(nx)
    j = np.arange(ny)
    k = np.arange(nz)
    fx = np.cos(math.pi * a * (i + 0.5) / nx) if walls[0] else np.cos(2 * math.pi * a * i / nx + 0.3 * a)
    fy = np.cos(math.pi * b * (j + 0.5) / ny) if walls[1] else np.sin(2 * math.pi * b * j / ny + 0.5 + b)
    fz = np.cos(math.pi * c * (k + 0.5) / nz)
    phi_e = fz[:, None, None] * fy[None, :, None] * fx[None, None, :]
    lam = (_eig_lambda(a, nx, lx / nx, walls[0]) + _eig_lambda(b, ny, ly / ny, walls[1])
           + _eig_lambda(c, 2 * nz, lz / nz, False))       # Neumann z: 4/h^2 sin^2(pi c / 2nz)
    Lphi = O.laplacian(g, phi_e)
    assert rel(Lphi, lam * phi_e) < 1e-12
    phi, _ = O.poisson(g, lam * phi_e)
    assert rel(phi, phi_e - vmean(g, phi_e)) < TOL


@pytest.mark.parametrize("beta", [0.0, 2.0, 3.0])
def test_solver_inverts_stencil_random(beta):
    """For a random mean-zero phi, S^-1 (L phi) = phi on stretched z."""
    nx, ny, nz = 12, 8, 16
    g = O.Grid(nx, ny, nz, lx=2 * math.pi, ly=2 * math.pi, lz=2.0, beta=beta)
    phi = synth.uniform_np(9, 1, (nz, ny, nx))
    phi -= vmean(g, phi)
    out, compat = O.poisson(g, O.laplacian(g, phi))
    assert rel(out, phi) < TOL
    assert abs(compat) < 1e-10 * np.max(np.abs(O.laplacian(g, phi)))


def test_manufactured_stretched():
    """Config-2 style: p = cos(3x)cos(5y)cos(pi z/2) on tanh-stretched z, RHS = L_h p."""
    nx, ny, nz = 32, 32, 24
    g = O.Grid(nx, ny, nz, lx=2 * math.pi, ly=2 * math.pi, lz=2.0, beta=2.0)
    x = np.arange(nx) * g.lx / nx + 0.5 * g.lx / nx
    y = np.arange(ny) * g.ly / ny + 0.5 * g.ly / ny
    zc = 0.5 * (g.zf[1:] + g.zf[:-1])
    p = np.cos(math.pi * zc / 2)[:, None, None] * np.cos(5 * y)[None, :, None] * np.cos(3 * x)[None, None, :]
    phi, _ = O.poisson(g, O.laplacian(g, p))
    assert rel(phi, p - vmean(g, p)) < TOL


def test_second_order_convergence():
    """Continuous RHS -(9+25+pi^2/4) p: error against p falls ~4x per halving of h."""
    errs = []
    for n in (16, 32, 64):
        g = O.Grid(n, n, n // 2, lx=2 * math.pi, ly=2 * math.pi, lz=2.0, beta=0.0)
        x = (np.arange(n) + 0.5) * g.lx / n
        zc = 0.5 * (g.zf[1:] + g.zf[:-1])
        p = np.cos(math.pi * zc / 2)[:, None, None] * np.cos(5 * x)[None, :, None] * np.cos(3 * x)[None, None, :]
        f = -(9 + 25 + math.pi ** 2 / 4) * p
        phi, _ = O.poisson(g, f)
        errs.append(np.max(np.abs(phi - (p - vmean(g, p)))))
    r1, r2 = errs[0] / errs[1], errs[1] / errs[2]
    assert 3.6 < r1 < 4.4 and 3.8 < r2 < 4.2, errs


def test_one_dimensional_column_by_cumsum():
    """nx = ny = 1: the Neumann problem is solved by two cumulative sums
    (flux F_{k+1} = F_k + hz_k b_k with F_0 = 0, then phi_k = phi_{k-1} + gz_k F_k)."""
    nz = 40
    g = O.Grid(1, 1, nz, lx=1.0, ly=1.0, lz=2.0, beta=2.5)
    b = synth.uniform_np(5, 1, (nz, 1, 1))
    b -= vmean(g, b)
    phi, _ = O.poisson(g, b)
    hz = g.hz
    zc = 0.5 * (g.zf[1:] + g.zf[:-1])
    F = np.concatenate([[0.0], np.cumsum(hz * b[:, 0, 0])])       # F at faces 0..nz
    ref = np.zeros(nz)
    for k in range(1, nz):
        ref[k] = ref[k - 1] + (zc[k] - zc[k - 1]) * F[k]
    ref -= np.sum(hz * ref) / np.sum(hz)
    assert abs(F[-1]) < 1e-12
    assert rel(phi[:, 0, 0], ref) < TOL


# ---------------------------------------------------------------- transforms
@pytest.mark.parametrize("n", [1, 2, 3, 5, 6, 8, 12, 16, 96])
def test_naive_dft_against_numpy(n):
    rng = np.random.default_rng(n)
    x = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    assert np.max(np.abs(O.dft(x) - np.fft.fft(x))) < 1e-12 * n
    assert np.max(np.abs(O.dft(x, inverse=True) - np.fft.ifft(x))) < 1e-12
    if n > 1:
        scipy_fft = pytest.importorskip("scipy.fft")
        xr = rng.standard_normal(n)
        # scipy's unnormalised DCT-II is 2 sum f_n cos(pi m (2n+1)/(2N))
        assert np.max(np.abs(O.dft(xr, dct=True).real - scipy_fft.dct(xr, type=2) / 2)) < 1e-12 * n
        assert np.max(np.abs(O.dft(O.dft(xr, dct=True), inverse=True, dct=True).real - xr)) < 1e-12


# ---------------------------------------------------------------- invariants
def _setup(nx=12, ny=8, nz=10, beta=2.0, seed=0):
    g = O.Grid(nx, ny, nz, lx=2 * math.pi, ly=math.pi, lz=2.0, beta=beta)
    return g, synth.uniform_velocity_np(seed, nx, ny, nz)


def test_divergence_free_and_idempotent():
    g, (u, v, w) = _setup()
    phi, u1, v1, w1, st = O.project(g, u, v, w)
    assert st[0] <= 1e-12 * st[1]
    phi2, u2, v2, w2, st2 = O.project(g, u1, v1, w1)
    assert np.max(np.abs(u2 - u1)) < 1e-12 and np.max(np.abs(w2 - w1)) < 1e-12
    assert np.max(np.abs(phi2)) < 1e-9 * np.max(np.abs(phi))
    # wall-normal velocity untouched, weighted mean of phi zero
    assert np.array_equal(w1[0], w[0]) and np.array_equal(w1[-1], w[-1])
    assert abs(vmean(g, phi)) < 1e-12 * np.max(np.abs(phi))


def test_linearity_and_alpha_dt_invariance():
    g, (u, v, w) = _setup(seed=1)
    _, (a, b, c) = _setup(seed=2)
    p1, u1, v1, w1, _ = O.project(g, u, v, w, dt=1e-3)
    p2, u2, v2, w2, _ = O.project(g, a, b, c, dt=1e-3)
    p3, u3, v3, w3, _ = O.project(g, 2 * u - a, 2 * v - b, 2 * w - c, dt=1e-3)
    assert rel(p3, 2 * p1 - p2) < 1e-12 and rel(u3, 2 * u1 - u2) < 1e-12
    # u_{n+1} does not depend on alpha dt; alpha dt phi does not either.  The
    # alpha values are the paper's printed RK/AB-CN coefficients.
    rows = [l.split() for l in open(__file__.replace("test_oracle_pins.py", "golden/rk_alpha.txt"))
            if l.strip() and not l.startswith("#")]
    alphas = sorted({Fraction(r[2]) + Fraction(r[3]) for r in rows})
    assert alphas == sorted([Fraction(1, 2), Fraction(8, 15), Fraction(2, 15), Fraction(1, 3), Fraction(1)])
    for al in map(float, alphas):
        pa, ua, va, wa, _ = O.project(g, u, v, w, dt=2e-3, alpha=al)
        assert rel(ua, u1) < 1e-12 and rel(wa, w1) < 1e-12
        assert rel(pa * al * 2e-3, p1 * 1e-3) < 1e-12


def test_translation_equivariance_and_mirror():
    g, (u, v, w) = _setup(seed=3)
    phi, u1, v1, w1, _ = O.project(g, u, v, w)
    # roll by 3 cells in x and 2 in y
    sh = lambda f: np.roll(np.roll(f, 3, axis=2), 2, axis=1)
    p2, u2, v2, w2, _ = O.project(g, sh(u), sh(v), sh(w))
    assert rel(p2, sh(phi)) < 1e-12 and rel(u2, sh(u1)) < 1e-12
    # symmetric tanh stretching: mirror z (w changes sign and swaps faces)
    p3, u3, v3, w3, _ = O.project(g, u[::-1], v[::-1], -w[::-1])
    assert rel(p3, phi[::-1]) < 1e-12 and rel(w3, -w1[::-1]) < 1e-12


def test_orthogonality_to_gradients():
    """<P u, G psi>_{V_f} = 0 for any psi (discrete Gauss: D = -V^-1 G^T V_f)."""
    g, (u, v, w) = _setup(seed=4)
    _, u1, v1, w1, _ = O.project(g, u, v, w)
    psi = synth.uniform_np(11, 1, g.cshape)
    gu, gv, gw = O.gradient(g, psi)
    dx, dy = g.lx / g.nx, g.ly / g.ny
    hz = g.hz
    zc = 0.5 * (g.zf[1:] + g.zf[:-1])
    gzf = np.zeros(g.nz + 1)
    gzf[1:-1] = np.diff(zc)
    ip = np.sum(u1 * gu * (dx * dy * hz)[:, None, None]) + np.sum(v1 * gv * (dx * dy * hz)[:, None, None]) \
        + np.sum(w1 * gw * (dx * dy * gzf)[:, None, None])
    scale = np.sqrt(np.sum(u1 ** 2) * np.sum(gu ** 2)) * dx * dy
    assert abs(ip) < 1e-12 * scale


# ---------------------------------------------------------------- adjoint
def test_adjoint_dot_product():
    g, (u, v, w) = _setup(nx=8, ny=12, nz=10, seed=5)
    wu = synth.normal_np(6, 1, u.shape)
    wv = synth.normal_np(6, 2, v.shape)
    ww = synth.normal_np(6, 3, w.shape)
    wp = synth.normal_np(6, 4, g.cshape)
    phi, u1, v1, w1, _ = O.project(g, u, v, w, dt=1e-3)
    lhs = np.sum(wu * u1) + np.sum(wv * v1) + np.sum(ww * w1) + np.sum(wp * phi)
    a, b, c = O.project_adjoint(g, wu, wv, ww, wp, dt=1e-3)
    rhs = np.sum(a * u) + np.sum(b * v) + np.sum(c * w)
    assert abs(lhs - rhs) < 1e-12 * (abs(lhs) + np.sqrt(np.sum(wp * wp) * np.sum(phi * phi)))


@pytest.mark.parametrize("walls", [(False, False), (True, False)])
def test_adjoint_matches_dense_transpose(walls):
    nx, ny, nz = 6, 8, 6
    g = O.Grid(nx, ny, nz, lx=1.1, ly=0.9, lz=2.0, beta=2.0, wall_x=walls[0], wall_y=walls[1])
    su, sv, sw = g.shapes
    gu, gv, gw = (synth.normal_np(7, t, s) for t, s in ((1, su), (2, sv), (3, sw)))
    gp = synth.normal_np(7, 4, g.cshape)
    a, b, c = O.project_adjoint(g, gu, gv, gw, gp, dt=2e-3, alpha=0.5)
    dp = dense.DenseProjection(nx, ny, nz, 1.1, 0.9, g.zf, *walls)
    ad, bd, cd = dp.project_T(gu, gv, gw, gp, dt=2e-3, alpha=0.5)
    for x, y in ((a, ad), (b, bd), (c, cd)):
        assert rel(x, y) < 1e-11


# ---------------------------------------------------------------- grid map
def test_tanh_faces_properties():
    nz, lz = 512, 2.0
    for beta in (1.0, 2.0, 2.5):
        zf = O.zfaces_tanh(nz, lz, beta)
        assert zf[0] == 0.0 and zf[-1] == lz
        assert np.all(np.diff(zf) > 0)
        assert np.max(np.abs(zf + zf[::-1] - lz)) < 1e-14        # symmetric about lz/2
        assert abs(zf[nz // 2] - lz / 2) < 1e-15
        hz = np.diff(zf)
        # centre/wall spacing ratio tends to cosh(beta)^2 for large nz
        assert abs(hz[nz // 2] / hz[0] / math.cosh(beta) ** 2 - 1) < 0.03
    z0 = O.zfaces_tanh(64, 1.0, 0.0)
    z1 = O.zfaces_tanh(64, 1.0, 1e-6)
    assert np.max(np.abs(z1 - np.arange(65) / 64)) < 1e-10 and np.max(np.abs(z0 - np.arange(65) / 64)) < 1e-15


# ---------------------------------------------------------------- Eq. (pressure)
@pytest.mark.parametrize("walls", [(False, False), (True, True)])
def test_pressure_update_closed_form(walls):
    """p_{n+1} = p_n + phi - alpha dt/(2 Re) lap(phi): for a discrete eigenfunction phi
    (eigenvalue lam, uniform z) this is p_n + (1 - alpha dt lam/(2 Re)) phi exactly, and
    with inv_re = 0 it is p_n + phi."""
    nx, ny, nz, a, b, c = 12, 16, 8, 3, 2, 1
    lx, ly, lz = 1.1, 0.8, 1.5
    g = O.Grid(nx, ny, nz, lx=lx, ly=ly, lz=lz, beta=0.0, wall_x=walls[0], wall_y=walls[1])
    i, j, k = np.arange(nx), np.arange(ny), np.arange(nz)
    fx = np.cos(math.pi * a * (i + 0.5) / nx) if walls[0] else np.cos(2 * math.pi * a * i / nx)
    fy = np.cos(math.pi * b * (j + 0.5) / ny) if walls[1] else np.cos(2 * math.pi * b * j / ny)
    fz = np.cos(math.pi * c * (k + 0.5) / nz)
    phi = fz[:, None, None] * fy[None, :, None] * fx[None, None, :]
    lam = (_eig_lambda(a, nx, lx / nx, walls[0]) + _eig_lambda(b, ny, ly / ny, walls[1])
           + _eig_lambda(c, 2 * nz, lz / nz, False))
    p_n = synth.normal_np(9, 1, phi.shape)
    dt, alpha, inv_re = 2e-3, 0.5, 1.0 / 40.0
    got = O.pressure_update(g, p_n, phi, dt, alpha, inv_re)
    assert rel(got, p_n + (1.0 - 0.5 * alpha * dt * inv_re * lam) * phi) < 1e-13
    assert np.array_equal(O.pressure_update(g, p_n, phi, dt, alpha, 0.0), p_n + phi)


# ---------------------------------------------------------------- Dirichlet outlet (phi = 0 at z = lz)
@pytest.mark.parametrize("shape,beta,walls", [
    ((8, 8, 8), 2.0, (False, False)), ((6, 12, 5), 0.0, (False, False)), ((6, 4, 7), 1.5, (True, True)),
    ((1, 1, 9), 2.5, (False, False)),
])
def test_dirichlet_outlet_matches_dense_solve(shape, beta, walls):
    """No compatibility mean, no reference value: phi solves L phi = D u*/(alpha dt)
    exactly (dense LU of the nonsingular L), and the top face velocity is corrected."""
    nx, ny, nz = shape
    g = O.Grid(nx, ny, nz, lx=1.3, ly=0.7, lz=2.0, beta=beta, wall_x=walls[0], wall_y=walls[1],
               dirichlet_top=True)
    u, v, w = synth.uniform_velocity_np(8, nx, ny, nz, *walls, zero_walls=False)
    phi, uu, vv, ww, st = O.project(g, u, v, w, dt=1e-3, alpha=1.0)
    dp = dense.DenseProjection(nx, ny, nz, 1.3, 0.7, g.zf, *walls, dirichlet_top=True)
    phid, ud, vd, wd = dp.project(u, v, w, dt=1e-3, alpha=1.0)
    assert rel(phi, phid) < TOL
    for a, b in ((uu, ud), (vv, vd), (ww, wd)):
        assert np.max(np.abs(a - b)) < TOL * max(1.0, np.max(np.abs(b)))
    assert st[2] == 0.0                                     # nothing removed
    assert st[0] <= 1e-10 * st[1]                           # divergence-free, incl. the top cells
    assert np.array_equal(ww[0], w[0])                      # the bottom wall is untouched
    assert not np.allclose(ww[-1], w[-1])                   # the outlet face is corrected


@pytest.mark.parametrize("a,b,c", [(0, 0, 0), (1, 2, 0), (0, 0, 3), (2, 1, 4)])
def test_dirichlet_outlet_eigenfunctions(a, b, c):
    """Uniform z, Neumann bottom and Dirichlet top: cos(pi (c+1/2)(k+1/2)/nz) is a discrete
    eigenfunction of the z second difference with eigenvalue -4/h^2 sin^2(pi (2c+1)/(4 nz))
    (the continued cosine vanishes on the top face, so its mirror value is -phi_{nz-1}).
    The (0,0,0) mode is regular here: the solver must return it, without mean removal."""
    nx, ny, nz = 12, 8, 10
    lx, ly, lz = 1.1, 0.9, 1.6
    g = O.Grid(nx, ny, nz, lx=lx, ly=ly, lz=lz, beta=0.0, dirichlet_top=True)
    i, j, k = np.arange(nx), np.arange(ny), np.arange(nz)
    fx = np.cos(2 * math.pi * a * i / nx)
    fy = np.cos(2 * math.pi * b * j / ny)
    fz = np.cos(math.pi * (c + 0.5) * (k + 0.5) / nz)
    phi_e = fz[:, None, None] * fy[None, :, None] * fx[None, None, :]
    hz = lz / nz
    lam = (_eig_lambda(a, nx, lx / nx, False) + _eig_lambda(b, ny, ly / ny, False)
           - 4.0 / hz ** 2 * math.sin(math.pi * (2 * c + 1) / (4 * nz)) ** 2)
    assert rel(O.laplacian(g, phi_e), lam * phi_e) < 1e-12
    phi, compat = O.poisson(g, lam * phi_e)
    assert compat == 0.0
    assert rel(phi, phi_e) < TOL


def test_dirichlet_outlet_adjoint_matches_dense_transpose():
    nx, ny, nz = 6, 4, 6
    g = O.Grid(nx, ny, nz, lx=1.1, ly=0.9, lz=2.0, beta=2.0, dirichlet_top=True)
    su, sv, sw = g.shapes
    gu, gv, gw = (synth.normal_np(17, t, s) for t, s in ((1, su), (2, sv), (3, sw)))
    gp = synth.normal_np(17, 4, g.cshape)
    a, b, c = O.project_adjoint(g, gu, gv, gw, gp, dt=2e-3, alpha=0.5)
    dp = dense.DenseProjection(nx, ny, nz, 1.1, 0.9, g.zf, dirichlet_top=True)
    ad, bd, cd = dp.project_T(gu, gv, gw, gp, dt=2e-3, alpha=0.5)
    for x, y in ((a, ad), (b, bd), (c, cd)):
        assert rel(x, y) < 1e-11


# ---------------------------------------------------------------- mass source q (Eq. elliptic)
def test_mass_source_closed_form_and_equivalence():
    """u* = 0 with q = -alpha dt lam phi_e (phi_e a discrete eigenfunction) gives phi = phi_e and
    u = -alpha dt G phi_e; and a source q = D e acts exactly like removing e from u*."""
    nx, ny, nz, a, b, c = 12, 8, 10, 2, 1, 3
    lx, ly, lz = 1.2, 0.8, 1.5
    g = O.Grid(nx, ny, nz, lx=lx, ly=ly, lz=lz, beta=0.0)
    i, j, k = np.arange(nx), np.arange(ny), np.arange(nz)
    phi_e = (np.cos(math.pi * c * (k + 0.5) / nz)[:, None, None] * np.cos(2 * math.pi * b * j / ny)[None, :, None]
             * np.cos(2 * math.pi * a * i / nx)[None, None, :])
    lam = (_eig_lambda(a, nx, lx / nx, False) + _eig_lambda(b, ny, ly / ny, False)
           + _eig_lambda(c, 2 * nz, lz / nz, False))
    dt, alpha = 2e-3, 0.5
    z = [np.zeros(s) for s in g.shapes]
    phi, u, v, w, compat = O.project_q(g, *z, -alpha * dt * lam * phi_e, dt=dt, alpha=alpha)
    assert rel(phi, phi_e) < TOL
    gu, gv, gw = O.gradient(g, phi_e)
    assert rel(u, -alpha * dt * gu) < 1e-11 and rel(w, -alpha * dt * gw) < 1e-11
    # equivalence with a shifted velocity, on a stretched grid
    g2 = O.Grid(8, 6, 7, lx=1.0, ly=0.7, lz=2.0, beta=2.0)
    us = synth.uniform_velocity_np(81, 8, 6, 7)
    e = synth.uniform_velocity_np(82, 8, 6, 7)
    q = O.divergence(g2, *e)
    phi_q, *_ = O.project_q(g2, *us, q, dt=dt, alpha=alpha)
    phi_s, *_ = O.project(g2, *(x - y for x, y in zip(us, e)), dt=dt, alpha=alpha)
    assert rel(phi_q, phi_s) < TOL

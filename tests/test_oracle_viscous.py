"""Pins of the viscous-solve oracle (oracle/viscous.py) to facts outside itself:
the FFT diagonalisation of periodic (circulant) operators, the discrete sine
eigenvectors of the wall-bounded second differences on a uniform grid, the
self-adjointness of the stretched operators in their volume weights, and a dense
Kronecker-product solve of the whole factored operator on tiny grids."""
import numpy as np
import pytest

from oracle import viscous as V


def rng(seed):
    return np.random.default_rng(seed)


@pytest.mark.parametrize("n", [1, 2, 3, 4, 7, 16, 33])
def test_periodic_solve_matches_fft_diagonalisation(n):
    # (I - beta L) is circulant: its eigenvalues are 1 + beta (4/h^2) sin^2(pi m / n)
    h, beta = 0.37, 0.8
    d = rng(n).standard_normal((3, 5, n))
    lam = 1.0 + beta * 4.0 / h ** 2 * np.sin(np.pi * np.arange(n) / n) ** 2
    ref = np.real(np.fft.ifft(np.fft.fft(d, axis=-1) / lam, axis=-1))
    got = V.periodic_solve(d, h, beta)
    assert np.abs(got - ref).max() <= 1e-13 * np.abs(ref).max()


def test_cyclic_thomas_general_corners_matches_dense():
    # Sherman-Morrison with distinct coefficients and corners, against LAPACK
    n = 9
    r = rng(3)
    sub, sup = r.uniform(-1, 0, n), r.uniform(-1, 0, n)
    diag = 3.0 + r.uniform(0, 1, n)
    lo, hi = -0.4, -0.7
    A = np.diag(diag) + np.diag(sub[1:], -1) + np.diag(sup[:-1], 1)
    A[n - 1, 0] = lo
    A[0, n - 1] = hi
    d = r.standard_normal((4, n))
    got = V.cyclic_thomas(sub, diag, sup, lo, hi, d)
    ref = np.linalg.solve(A, d.T).T
    assert np.abs(got - ref).max() <= 1e-13 * np.abs(ref).max()


@pytest.mark.parametrize("nz", [1, 2, 5, 16])
def test_cell_operator_sine_eigenvectors_uniform(nz):
    # Dirichlet at the wall faces, unknowns at the centres: DST-II vectors
    # sin(pi l (k + 1/2) / nz), eigenvalues -(4/h^2) sin^2(pi l / (2 nz)), l = 1..nz
    lz_len = 1.7
    zf = np.linspace(0.0, lz_len, nz + 1)
    h = lz_len / nz
    beta = 0.03
    k = np.arange(nz)
    for l in range(1, nz + 1):
        s = np.sin(np.pi * l * (k + 0.5) / nz)
        lam = -4.0 / h ** 2 * np.sin(np.pi * l / (2 * nz)) ** 2
        got = V.z_solve(s, V.lz_cell(zf), beta)
        assert np.abs(got - s / (1.0 - beta * lam)).max() <= 1e-13


@pytest.mark.parametrize("nz", [2, 3, 6, 17])
def test_face_operator_sine_eigenvectors_uniform(nz):
    # zero wall faces, unknowns at the interior faces: DST-I vectors sin(pi l k / nz)
    lz_len = 2.0
    zf = np.linspace(0.0, lz_len, nz + 1)
    h = lz_len / nz
    beta = 0.05
    k = np.arange(1, nz)
    for l in range(1, nz):
        s = np.sin(np.pi * l * k / nz)
        lam = -4.0 / h ** 2 * np.sin(np.pi * l / (2 * nz)) ** 2
        got = V.z_solve(s, V.lz_face(zf), beta)
        assert np.abs(got - s / (1.0 - beta * lam)).max() <= 1e-12


def tri(lz):
    sub, diag, sup = lz
    n = len(diag)
    return np.diag(diag) + np.diag(sub[1:], -1) + np.diag(sup[:-1], 1) if n else np.zeros((0, 0))


def stretched(nz, beta_map=2.0, lz_len=2.0):
    k = np.arange(nz + 1)
    zf = 0.5 * lz_len * (1.0 + np.tanh(beta_map * (2.0 * k / nz - 1.0)) / np.tanh(beta_map))
    zf[0], zf[-1] = 0.0, lz_len
    return zf


@pytest.mark.parametrize("nz", [3, 8, 21])
def test_stretched_operators_self_adjoint_in_volume_weights(nz):
    # <f, L g>_W = <L f, g>_W with W = cell heights (centres) or centre spacings (faces):
    # a wrong metric (a swapped hz / dzc, a missing factor 2 at the wall) breaks it
    zf = stretched(nz)
    hz = np.diff(zf)
    zc = 0.5 * (zf[1:] + zf[:-1])
    Lc = tri(V.lz_cell(zf))
    assert np.abs(np.diag(hz) @ Lc - (np.diag(hz) @ Lc).T).max() <= 1e-12 * np.abs(Lc).max() * hz.max()
    Lf = tri(V.lz_face(zf))
    wf = np.diff(zc)
    assert np.abs(np.diag(wf) @ Lf - (np.diag(wf) @ Lf).T).max() <= 1e-12 * np.abs(Lf).max() * wf.max()
    # negative definite (a sign error in the wall terms would break it)
    assert np.linalg.eigvalsh(0.5 * (np.diag(hz) @ Lc + (np.diag(hz) @ Lc).T)).max() < 0


def test_cell_operator_row_sums_are_the_wall_fluxes():
    # on a stretched grid the centre operator applied to f = 1 gives the wall flux only:
    # interior rows sum to zero, the first row is -2 / hz_0^2 (mirror ghost at distance hz_0)
    zf = stretched(6)
    hz = np.diff(zf)
    Lc = tri(V.lz_cell(zf))
    s = Lc.sum(axis=1)
    assert np.abs(s[1:-1]).max() <= 1e-9 * np.abs(Lc).max()
    assert s[0] == pytest.approx(-2.0 / hz[0] ** 2, rel=1e-13)
    assert s[-1] == pytest.approx(-2.0 / hz[-1] ** 2, rel=1e-13)


def test_beta_zero_is_identity():
    nx, ny, nz = 5, 4, 3
    zf = stretched(nz)
    r = rng(9)
    ru, rv, rw = r.standard_normal((nz, ny, nx)), r.standard_normal((nz, ny, nx)), r.standard_normal((nz + 1, ny, nx))
    du, dv, dw = V.viscous_solve(nx, ny, nz, 1.0, 2.0, zf, ru, rv, rw, 0.0)
    assert np.array_equal(du, ru) and np.array_equal(dv, rv)
    assert np.array_equal(dw[1:nz], rw[1:nz]) and not dw[0].any() and not dw[nz].any()


def periodic_matrix(n, h, beta):
    s = beta / h ** 2
    A = np.eye(n) * (1.0 + 2.0 * s)
    for i in range(n):
        A[i, (i + 1) % n] -= s
        A[i, (i - 1) % n] -= s
    return A


@pytest.mark.parametrize("shape", [(4, 3, 5), (6, 5, 4), (3, 7, 2), (1, 2, 3)])
def test_factored_solve_matches_dense_kronecker(shape):
    # the factored operator as one dense matrix kron(Hz, Hy, Hx) ([k][j][i] order), solved
    # by LAPACK: pins the axes (dx != dy), the order-independence and every wall term
    nx, ny, nz = shape
    lx, ly, beta = 1.3, 0.7, 0.02
    zf = stretched(nz)
    Hx = periodic_matrix(nx, lx / nx, beta)
    Hy = periodic_matrix(ny, ly / ny, beta)
    r = rng(11)
    ru, rv, rw = r.standard_normal((nz, ny, nx)), r.standard_normal((nz, ny, nx)), r.standard_normal((nz + 1, ny, nx))
    du, dv, dw = V.viscous_solve(nx, ny, nz, lx, ly, zf, ru, rv, rw, beta)
    Hzc = np.eye(nz) - beta * tri(V.lz_cell(zf))
    Mc = np.kron(Hzc, np.kron(Hy, Hx))
    for got, rr in ((du, ru), (dv, rv)):
        ref = np.linalg.solve(Mc, rr.ravel()).reshape(rr.shape)
        assert np.abs(got - ref).max() <= 1e-12 * np.abs(ref).max()
    if nz > 1:
        Hzf = np.eye(nz - 1) - beta * tri(V.lz_face(zf))
        Mf = np.kron(Hzf, np.kron(Hy, Hx))
        ref = np.linalg.solve(Mf, rw[1:nz].ravel()).reshape(rw[1:nz].shape)
        assert np.abs(dw[1:nz] - ref).max() <= 1e-12 * np.abs(ref).max()
    assert not dw[0].any() and not dw[nz].any()


def test_fourier_mode_closed_form_3d():
    # rhs = cos(2 pi m x / lx) sin(2 pi n y / ly) * (z eigenvector): the solve scales it by
    # the product of the three 1-D eigenvalue factors
    nx, ny, nz = 16, 12, 8
    lx, ly, lz_len, beta = 2 * np.pi, 1.5, 2.0, 0.01
    zf = np.linspace(0.0, lz_len, nz + 1)
    dx, dy, h = lx / nx, ly / ny, lz_len / nz
    m, n, l = 3, 2, 4
    x = np.arange(nx) * dx
    y = (np.arange(ny) + 0.5) * dy
    k = np.arange(nz)
    f = np.sin(np.pi * l * (k + 0.5) / nz)[:, None, None] * np.sin(2 * np.pi * n * y / ly)[None, :, None] \
        * np.cos(2 * np.pi * m * x / lx)[None, None, :]
    fac = (1 + beta * 4 / dx ** 2 * np.sin(np.pi * m / nx) ** 2) * (1 + beta * 4 / dy ** 2 * np.sin(np.pi * n / ny) ** 2) \
        * (1 + beta * 4 / h ** 2 * np.sin(np.pi * l / (2 * nz)) ** 2)
    du, dv, _ = V.viscous_solve(nx, ny, nz, lx, ly, zf, f, f, np.zeros((nz + 1, ny, nx)), beta)
    assert np.abs(du - f / fac).max() <= 1e-13
    assert np.abs(dv - f / fac).max() <= 1e-13

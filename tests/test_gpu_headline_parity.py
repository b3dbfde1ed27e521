"""Parity with the FP64 oracle on the kernel path the benchmark runs.

At 1024 points per direction the two-level FFT takes the factor-32 register DFT on both
passes (1024 = 32 x 32); 768 = 32 x 24 and 512 = 32 x 16 take it on one.  The bench's
launch shape (x and y factors 32, streaming y/z kernels with one x-mode per column block,
which on the mixed path is the pipelined kernel pair, 16 rows per x CTA) is the default
for every 1024 x 1024 x nz grid, so a few z levels exercise it at a cost the oracle's naive
transforms can pay.  The solver is the paper's (Section "Fluid domain", projection
paragraph: FFTs in x1 and x2, one tridiagonal solve along x3 per mode) for Eq. (elliptic)
and Eq. (velsolen).

Tolerances as in test_gpu_parity: FP64 relative L2 of phi <= 1e-12, velocity <= 1e-11
max|u*|, max|D u| <= 1e-11 max|D u*|; mixed 1e-9 for all three.  On the stretched 1024^2
planes one refinement sweep meets the bound on phi but leaves the velocity and the
divergence at a few 1e-9 and 1e-8 (every fp32 transform rounds at 2^-24 of its plane's
norm, and the stencil amplifies the rounding of phi next to the walls); the second sweep
brings them to 1e-12 and 1e-10, so the mixed cases here run two sweeps (the count the
benchmark runs) and the one-sweep result is held to the bound on phi.
"""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import oracle as O  # noqa: E402
from paper_2609_19130_gb300 import FP64, MIXED, Grid, Plan, synth  # noqa: E402
from paper_2609_19130_gb300 import _native as N  # noqa: E402

pytestmark = pytest.mark.gpu

TOL = {FP64: dict(phi=1e-12, u=1e-11, div=1e-11), MIXED: dict(phi=1e-9, u=1e-9, div=1e-9)}
# the launch shape bench.py times at 1024 x 1024 x 512
BENCH_SHAPE = {MIXED: dict(rows=16, x_n1=32, y_n1=32, yz_kernel=1, mb=1),
               FP64: dict(rows=8, x_n1=32, y_n1=32, yz_kernel=1, mb=2)}


@pytest.fixture(scope="module", autouse=True)
def _build():
    from paper_2609_19130_gb300 import build
    build.build()


def rel_l2(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def run_gpu(grid, prec, refine, fields, dt, alpha=1.0, shape=None):
    plan = Plan([grid], precision=prec, refine_steps=refine)
    tun = plan.tuning(0)
    if shape is not None:
        for k, val in shape.items():
            assert tun[k] == val, (k, tun)
    t = [x if torch.is_tensor(x) else torch.from_numpy(np.ascontiguousarray(x)).cuda() for x in fields]
    (uo, vo, wo, po), st = plan.project(*t, dt, alpha, stats=True)
    torch.cuda.synchronize()
    status = plan.sync_status()
    plan.close()
    return [x.cpu().numpy() for x in (uo, vo, wo, po)], {k: float(v.cpu()[0]) for k, v in st.items()}, status


def compare(grid, og, prec, refine, fields_np, fields_dev, oracle_out, dt, alpha=1.0, shape=None):
    phi_o, u_o, v_o, w_o, st_o = oracle_out
    (ug, vg, wg, pg), st, status = run_gpu(grid, prec, refine, fields_dev, dt, alpha, shape)
    t = TOL[prec]
    umax = max(np.abs(a).max() for a in fields_np)
    assert status == 0, status
    e_phi = rel_l2(pg, phi_o)
    assert e_phi <= t["phi"], e_phi
    for a, b in ((ug, u_o), (vg, v_o), (wg, w_o)):
        assert np.abs(a - b).max() <= t["u"] * umax, np.abs(a - b).max() / umax
    w_in = fields_np[2]
    assert np.array_equal(wg[0], w_in[0]) and np.array_equal(wg[-1], w_in[-1])
    assert st["max_div"] <= t["div"] * st_o[1], (st["max_div"], st_o[1])
    # the library's max|D u*| is the fp32 maximum of |b| (the statistic is for reporting)
    assert abs(st["max_div_in"] - st_o[1]) <= 1e-6 * st_o[1]
    return pg, e_phi


# ------------------------------------------------------------------ bench recipe at 8 levels
@pytest.fixture(scope="module")
def bench_recipe_8():
    nx, ny, nz, beta = 1024, 1024, 8, 2.5
    g = Grid(nx, ny, nz, 2 * math.pi, 2 * math.pi, 2.0, beta=beta)
    dev = synth.kolmogorov_velocity_torch(4, nx, ny, nz, torch.device("cuda"))
    host = [x.cpu().numpy() for x in dev]
    og = O.Grid(nx, ny, nz, lx=g.lx, ly=g.ly, lz=2.0, beta=beta)
    return g, og, dev, host, O.project(og, *host, dt=1e-3)


@pytest.mark.parametrize("prec,refine", [(FP64, 0), (MIXED, 2)])
def test_bench_recipe_1024x1024x8(bench_recipe_8, prec, refine):
    """The bench's workload (k^-5/3 velocity of seed 4, tanh 2.5, 2 pi x 2 pi x [0, 2]) on 8
    levels, in the bench's launch shape: element-wise against the oracle."""
    g, og, dev, host, ref = bench_recipe_8
    compare(g, og, prec, refine, host, dev, ref, 1e-3, shape=BENCH_SHAPE[prec])


def test_bench_recipe_1024x1024x8_one_sweep_phi(bench_recipe_8):
    """One refinement sweep on the same grid and launch shape: phi within the stated 1e-9."""
    g, og, dev, host, ref = bench_recipe_8
    (_, _, _, pg), _, status = run_gpu(g, MIXED, 1, dev, 1e-3, shape=BENCH_SHAPE[MIXED])
    assert status == 0
    assert rel_l2(pg, ref[0]) <= 1e-9


# ------------------------------------------------------------------ mixed factor-32 transforms
@pytest.fixture(scope="module")
def grid_768x512():
    nx, ny, nz = 768, 512, 6
    g = Grid(nx, ny, nz, 2 * math.pi, 1.7, 2.0, beta=2.0)
    host = synth.uniform_velocity_np(23, nx, ny, nz)
    og = O.Grid(nx, ny, nz, lx=g.lx, ly=g.ly, lz=2.0, beta=2.0)
    return g, og, host, O.project(og, *host, dt=2e-3, alpha=0.5)


@pytest.mark.parametrize("prec,refine", [(FP64, 0), (MIXED, 2)])
def test_768x512x6_factor32(grid_768x512, prec, refine):
    """768 = 32 x 24 along x and 512 = 32 x 16 along y, U[-1,1] velocity."""
    g, og, host, ref = grid_768x512
    shape = dict(x_n1=32, y_n1=32)
    compare(g, og, prec, refine, host, host, ref, 2e-3, 0.5, shape=shape)


@pytest.mark.parametrize("prec,refine", [(FP64, 0), (MIXED, 1)])
def test_wall_x_512_dct(prec, refine):
    """A wall-bounded x of 512 cells: DCT-II through a 512-point (32 x 16) FFT, with ny = 1024
    (32 x 32) along y."""
    nx, ny, nz = 512, 1024, 4
    g = Grid(nx, ny, nz, 1.0, 2.0, 1.0, beta=1.5, bc_x=N.IBF_BC_NEUMANN)
    host = synth.uniform_velocity_np(29, nx, ny, nz, wall_x=True)
    og = O.Grid(nx, ny, nz, lx=1.0, ly=2.0, lz=1.0, beta=1.5, wall_x=True)
    ref = O.project(og, *host, dt=1e-3)
    pg, _ = compare(g, og, prec, refine, host, host, ref, 1e-3, shape=dict(x_n1=32, y_n1=32))


# ------------------------------------------------------------------ config 2 at its stated size
def manufactured(nx, ny, nz, lx, ly, zf):
    x = (np.arange(nx) + 0.5) * lx / nx
    y = (np.arange(ny) + 0.5) * ly / ny
    zc = 0.5 * (zf[1:] + zf[:-1])
    return np.cos(math.pi * zc / 2)[:, None, None] * np.cos(5 * y)[None, :, None] * np.cos(3 * x)[None, None, :]


@pytest.fixture(scope="module")
def config2_full():
    n, dt = 256, 1e-3
    g = Grid(n, n, n, 2 * math.pi, 2 * math.pi, 2.0, beta=2.0)
    og = O.Grid(n, n, n, lx=g.lx, ly=g.ly, lz=2.0, beta=2.0)
    u, v, w = synth.uniform_velocity_np(2, n, n, n)
    pm = manufactured(n, n, n, g.lx, g.ly, og.zf)
    gu, gv, gw = O.gradient(og, pm)
    star = (u + dt * gu, v + dt * gv, w + dt * gw)
    return g, og, (u, v, w), star, pm, O.project(og, *star, dt=dt)


@pytest.mark.parametrize("prec,refine", [(FP64, 0), (MIXED, 1)])
def test_config2_256cube_oracle_and_manufactured(config2_full, prec, refine):
    """Config 2 at 256^3: U[-1,1] velocity of seed 2 plus alpha dt G p_m with
    p_m = cos 3x cos 5y cos(pi z/2) on the tanh-2 grid; element-wise against the oracle, and
    the GPU recovers p_m (minus its weighted mean) as the difference of the solves with and
    without the manufactured part."""
    g, og, base, star, pm, ref = config2_full
    pg, _ = compare(g, og, prec, refine, star, star, ref, 1e-3)
    (_, _, _, pb), _, status = run_gpu(g, prec, refine, base, 1e-3)
    assert status == 0
    V = og.hz[:, None, None]
    pm0 = pm - np.sum(V * pm) / (np.sum(V) * g.nx * g.ny)
    # phi of the two solves each carry the solve's error (bounded above); their difference
    # is p_m to within the sum of the two
    bound = 2 * TOL[prec]["phi"] * np.linalg.norm(ref[0]) + 1e-13 * np.linalg.norm(pm0)
    assert np.linalg.norm((pg - pb) - pm0) <= bound, (np.linalg.norm((pg - pb) - pm0), bound)

"""Wall-bounded x and/or y (DCT-II transform, Neumann phi): CUDA path vs the FP64 oracle.

The paper's configurations are all periodic in x and y; a wall-bounded horizontal
direction is the library's extension (DCT-II through an FFT of the same length with
Makhoul's reordering and pre/post twiddles).  Same tolerances as the periodic parity
tests: FP64 relative L2 of phi <= 1e-12, mixed <= 1e-9 after one refinement sweep.
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
NEU = N.IBF_BC_NEUMANN


@pytest.fixture(scope="module", autouse=True)
def _build():
    from paper_2609_19130_gb300 import build
    build.build()


def rel_l2(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def cuda(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to("cuda")


def make(nx, ny, nz, wx, wy, beta, lx=2 * math.pi, ly=1.3, lz=2.0):
    g = Grid(nx, ny, nz, lx, ly, lz, beta=beta, bc_x=NEU if wx else 0, bc_y=NEU if wy else 0)
    og = O.Grid(nx, ny, nz, lx=lx, ly=ly, lz=lz, beta=beta, wall_x=wx, wall_y=wy)
    return g, og


def run(g, prec, u, v, w, dt, alpha):
    plan = Plan([g], precision=prec, refine_steps=1 if prec == MIXED else 0)
    (uo, vo, wo, po), st = plan.project(cuda(u), cuda(v), cuda(w), dt, alpha, stats=True)
    torch.cuda.synchronize()
    status = plan.sync_status()
    plan.close()
    return [x.cpu().numpy() for x in (uo, vo, wo, po)], {k: float(t.cpu()[0]) for k, t in st.items()}, status


# (nx, ny, nz, wall_x, wall_y, beta): several FFT tiles, ragged tails, odd DCT lengths
# (3, 9), length 1, and every wall combination
CASES = [
    (16, 12, 8, True, False, 2.0), (16, 12, 8, False, True, 2.0), (16, 12, 8, True, True, 2.0),
    (9, 6, 5, True, False, 1.0), (6, 9, 7, False, True, 1.5), (3, 3, 4, True, True, 0.0),
    (96, 64, 17, True, False, 2.5), (64, 96, 9, False, True, 2.5), (48, 24, 12, True, True, 3.0),
    (1, 16, 6, True, False, 1.0), (16, 1, 6, False, True, 1.0), (192, 32, 5, True, True, 2.0),
]


@pytest.mark.parametrize("case", CASES, ids=lambda c: "{}x{}x{}{}{}".format(*c[:3], "_wx" if c[3] else "",
                                                                          "_wy" if c[4] else ""))
@pytest.mark.parametrize("prec", [FP64, MIXED])
def test_walls_match_oracle(case, prec):
    nx, ny, nz, wx, wy, beta = case
    g, og = make(nx, ny, nz, wx, wy, beta)
    u, v, w = synth.uniform_velocity_np(23, nx, ny, nz, wall_x=wx, wall_y=wy)
    assert (u.shape, v.shape, w.shape) == g.shapes
    phi_o, u_o, v_o, w_o, st_o = O.project(og, u, v, w, dt=2e-3, alpha=0.7)
    (ug, vg, wg, pg), st, status = run(g, prec, u, v, w, 2e-3, 0.7)
    t = TOL[prec]
    umax = max(np.abs(u).max(), np.abs(v).max(), np.abs(w).max())
    assert status in (0, 7), status
    assert rel_l2(pg, phi_o) <= t["phi"], rel_l2(pg, phi_o)
    for a, b in ((ug, u_o), (vg, v_o), (wg, w_o)):
        assert np.abs(a - b).max() <= t["u"] * umax, np.abs(a - b).max()
    # wall faces keep the imposed normal velocity bit for bit
    if wx:
        assert np.array_equal(ug[:, :, 0], u[:, :, 0]) and np.array_equal(ug[:, :, -1], u[:, :, -1])
    if wy:
        assert np.array_equal(vg[:, 0, :], v[:, 0, :]) and np.array_equal(vg[:, -1, :], v[:, -1, :])
    assert np.array_equal(wg[0], w[0]) and np.array_equal(wg[-1], w[-1])
    assert st["max_div"] <= t["div"] * st_o[1], (st["max_div"], st_o[1])
    assert abs(st["max_div_in"] - st_o[1]) <= 1e-6 * st_o[1]


@pytest.mark.parametrize("prec", [FP64, MIXED])
def test_walls_nonzero_wall_flux(prec):
    """Inflow/outflow through the x and y walls: the compatibility defect is removed
    and reported exactly as the oracle does."""
    nx, ny, nz = 24, 16, 10
    g, og = make(nx, ny, nz, True, True, 1.5)
    u, v, w = synth.uniform_velocity_np(31, nx, ny, nz, wall_x=True, wall_y=True, zero_walls=False)
    phi_o, u_o, *_, st_o = O.project(og, u, v, w)
    (ug, vg, wg, pg), st, status = run(g, prec, u, v, w, 1e-3, 1.0)
    assert status == 7  # IBF_WARN_INCOMPATIBLE_RHS
    assert abs(st["compat"] - st_o[2]) <= 1e-9 * abs(st_o[2])
    assert rel_l2(pg, phi_o) <= TOL[prec]["phi"]
    assert np.abs(ug - u_o).max() <= TOL[prec]["u"] * np.abs(u).max()


def test_walls_dct_eigenfunction():
    """phi = cos(pi a (i+1/2)/nx) cos(pi b (j+1/2)/ny) cos(pi c (k+1/2)/nz) is an exact
    discrete eigenfunction of L with Neumann walls in x, y and z (uniform spacing):
    the projection of u* = alpha dt G phi returns phi itself (zero weighted mean)."""
    nx, ny, nz, a, b, c = 12, 16, 8, 3, 5, 2
    g, og = make(nx, ny, nz, True, True, 0.0, lx=1.0, ly=1.5, lz=2.0)
    i, j, k = np.arange(nx) + 0.5, np.arange(ny) + 0.5, np.arange(nz) + 0.5
    phi = (np.cos(math.pi * c * k / nz)[:, None, None] * np.cos(math.pi * b * j / ny)[None, :, None]
           * np.cos(math.pi * a * i / nx)[None, None, :])
    dt, alpha = 1e-3, 1.0
    gu, gv, gw = O.gradient(og, phi)
    u, v, w = alpha * dt * gu, alpha * dt * gv, alpha * dt * gw
    for prec in (FP64, MIXED):
        (ug, vg, wg, pg), st, status = run(g, prec, u, v, w, dt, alpha)
        assert rel_l2(pg, phi) <= TOL[prec]["phi"] * 10, rel_l2(pg, phi)
        assert np.abs(ug).max() <= 1e-9 * np.abs(u).max()


@pytest.mark.parametrize("prec,tol", [(FP64, 1e-11), (MIXED, 1e-8)])
@pytest.mark.parametrize("wx,wy", [(True, False), (False, True), (True, True)])
def test_walls_adjoint_matches_oracle(prec, tol, wx, wy):
    nx, ny, nz = 16, 12, 10
    g, og = make(nx, ny, nz, wx, wy, 2.0, lx=1.1, ly=0.9)
    su, sv, sw = g.shapes
    gu, gv, gw = (synth.normal_np(6, i + 1, s) for i, s in enumerate((su, sv, sw)))
    gp = synth.normal_np(6, 4, (nz, ny, nx))
    ref = O.project_adjoint(og, gu, gv, gw, gp, dt=2e-3, alpha=0.5)
    plan = Plan([g], precision=prec, refine_steps=1 if prec == MIXED else 0)
    a, b, c = (torch.empty(s, dtype=torch.float64, device="cuda") for s in (su, sv, sw))
    plan.backward_into([(cuda(gu), cuda(gv), cuda(gw), cuda(gp))], [(a, b, c)], 2e-3, 0.5)
    torch.cuda.synchronize()
    plan.close()
    for x, y in zip((a, b, c), ref):
        assert rel_l2(x.cpu().numpy(), y) <= tol, rel_l2(x.cpu().numpy(), y)


def test_batch_mixed_boundary_conditions():
    """One plan over grids with different horizontal boundary conditions."""
    draws = [(32, 24, 16, False, False, 1.3), (12, 48, 9, True, False, 2.7), (24, 12, 8, False, True, 1.0),
             (6, 6, 33, True, True, 2.0), (64, 32, 12, True, True, 2.5)]
    made = [make(nx, ny, nz, wx, wy, b) for nx, ny, nz, wx, wy, b in draws]
    fields = [synth.uniform_velocity_np(1000 + i, *d[:3], wall_x=d[3], wall_y=d[4]) for i, d in enumerate(draws)]
    for prec in (FP64, MIXED):
        plan = Plan([g for g, _ in made], precision=prec, refine_steps=1 if prec == MIXED else 0)
        outs = plan.project_batch([tuple(cuda(a) for a in f) for f in fields], 1e-3)
        torch.cuda.synchronize()
        for (g, og), f, o in zip(made, fields, outs):
            phi_o, uo, vo, wo, _ = O.project(og, *f)
            assert rel_l2(o[3].cpu().numpy(), phi_o) <= TOL[prec]["phi"]
            assert np.abs(o[0].cpu().numpy() - uo).max() <= TOL[prec]["u"]
            assert np.abs(o[1].cpu().numpy() - vo).max() <= TOL[prec]["u"]
        plan.close()

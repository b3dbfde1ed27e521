"""Parity of the CUDA projection (through the C ABI) with the FP64 oracle.

Tolerances (the fp64 bounds are rounding of O(10) transform and sweep operations on
values of size max|u*|; the mixed ones are the stated 1e-9, met after one refinement
sweep, which leaves an error of about (fp32 error)^2 of the solve):
  FP64 path : relative L2 of phi <= 1e-12, velocity max error <= 1e-11 max|u*|,
              max|D u| <= 1e-11 max|D u*|;
  mixed path: relative L2 of phi <= 1e-9 after refinement, velocity max error
              <= 1e-9 max|u*|, max|D u| <= 1e-9 max|D u*|.
"""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import oracle as O  # noqa: E402
from paper_2609_19130_gb300 import FP64, MIXED, Grid, Plan, Projection, synth  # noqa: E402

pytestmark = pytest.mark.gpu

TOL = {FP64: dict(phi=1e-12, u=1e-11, div=1e-11), MIXED: dict(phi=1e-9, u=1e-9, div=1e-9)}


@pytest.fixture(scope="module", autouse=True)
def _build():
    from paper_2609_19130_gb300 import build
    build.build()


def rel_l2(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def cuda(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to("cuda")


def gpu_project(grid, prec, refine, u, v, w, dt=1e-3, alpha=1.0):
    plan = Plan([grid], precision=prec, refine_steps=refine)
    (uo, vo, wo, po), st = plan.project(cuda(u), cuda(v), cuda(w), dt, alpha, stats=True)
    torch.cuda.synchronize()
    status = plan.sync_status()
    out = [x.cpu().numpy() for x in (uo, vo, wo, po)]
    plan.close()
    return out, {k: float(t.cpu()[0]) for k, t in st.items()}, status


def check_against_oracle(grid, prec, refine, u, v, w, dt=1e-3, alpha=1.0):
    og = O.Grid(grid.nx, grid.ny, grid.nz, lx=grid.lx, ly=grid.ly, lz=grid.lz, beta=grid.beta,
                zf=grid.zf)
    phi_o, u_o, v_o, w_o, st_o = O.project(og, u, v, w, dt=dt, alpha=alpha)
    (ug, vg, wg, pg), st, status = gpu_project(grid, prec, refine, u, v, w, dt, alpha)
    t = TOL[prec]
    umax = max(np.abs(u).max(), np.abs(v).max(), np.abs(w).max())
    assert status in (0, 7), status
    assert rel_l2(pg, phi_o) <= t["phi"], rel_l2(pg, phi_o)
    for a, b in ((ug, u_o), (vg, v_o), (wg, w_o)):
        assert np.abs(a - b).max() <= t["u"] * umax, np.abs(a - b).max()
    assert np.array_equal(wg[0], w[0]) and np.array_equal(wg[-1], w[-1])   # walls untouched
    assert st["max_div"] <= t["div"] * st_o[1], (st["max_div"], st_o[1])
    assert abs(st["max_div_in"] - st_o[1]) <= 1e-6 * st_o[1]
    return pg, phi_o


# ------------------------------------------------------------------ config 1
@pytest.mark.parametrize("prec,refine", [(FP64, 0), (MIXED, 1), (MIXED, 2)])
def test_config1_32cube(prec, refine):
    """32^3 periodic x,y, Neumann z, uniform unit box, dt = 1e-3, U[-1,1] seed 0, w* = 0 on walls."""
    g = Grid(32, 32, 32, 1.0, 1.0, 1.0, beta=0.0)
    u, v, w = synth.uniform_velocity_np(0, 32, 32, 32)
    check_against_oracle(g, prec, refine, u, v, w)


# ------------------------------------------------------------------ shapes: several tiles, ragged tails
SHAPES = [
    (8, 8, 8, 2.0), (6, 12, 8, 2.0), (12, 6, 5, 1.0), (96, 64, 17, 2.5), (1, 1, 12, 2.0),
    (32, 1, 9, 1.5), (1, 16, 7, 1.5), (24, 48, 33, 3.0), (192, 96, 20, 2.0), (64, 128, 3, 2.0),
    (16, 16, 1, 0.0),
]


@pytest.mark.parametrize("shape", SHAPES, ids=lambda s: "x".join(map(str, s[:3])))
@pytest.mark.parametrize("prec", [FP64, MIXED])
def test_shapes(shape, prec):
    nx, ny, nz, beta = shape
    g = Grid(nx, ny, nz, 2 * math.pi, 1.3, 2.0, beta=beta)
    u, v, w = synth.uniform_velocity_np(17, nx, ny, nz)
    check_against_oracle(g, prec, 1 if prec == MIXED else 0, u, v, w, dt=3e-3, alpha=0.5)


def test_explicit_faces_and_incompatible_rhs():
    nx, ny, nz = 16, 12, 10
    zf = np.cumsum(np.concatenate([[0.0], 0.5 + synth.uniform_np(3, 9, (nz,), 0.0, 1.0)]))
    zf = zf / zf[-1] * 1.7
    g = Grid(nx, ny, nz, 1.0, 2.0, 1.7, zf=zf)
    u, v, w = synth.uniform_velocity_np(4, nx, ny, nz, zero_walls=False)   # wall fluxes do not cancel
    for prec in (FP64, MIXED):
        og = O.Grid(nx, ny, nz, lx=1.0, ly=2.0, lz=1.7, zf=zf)
        phi_o, *_ , st_o = O.project(og, u, v, w)
        (ug, vg, wg, pg), st, status = gpu_project(g, prec, 1 if prec == MIXED else 0, u, v, w)
        assert status == 7      # IBF_WARN_INCOMPATIBLE_RHS
        assert abs(st["compat"] - st_o[2]) <= 1e-9 * abs(st_o[2])
        assert rel_l2(pg, phi_o) <= TOL[prec]["phi"]


# ------------------------------------------------------------------ config 2 (reduced size, element-wise)
def manufactured(g):
    x = (np.arange(g.nx) + 0.5) * g.lx / g.nx
    y = (np.arange(g.ny) + 0.5) * g.ly / g.ny
    zf = O.zfaces_tanh(g.nz, g.lz, g.beta)
    zc = 0.5 * (zf[1:] + zf[:-1])
    return np.cos(math.pi * zc / 2)[:, None, None] * np.cos(5 * y)[None, :, None] * np.cos(3 * x)[None, None, :]


@pytest.mark.parametrize("prec,refine", [(FP64, 0), (MIXED, 1)])
def test_config2_manufactured_reduced(prec, refine):
    """Config 2 recipe at 64^3: periodic 2 pi x 2 pi, z in [0,2] tanh beta=2, U[-1,1] seed 2
    plus alpha dt G p_m so that phi contains p_m exactly."""
    n, dt = 64, 1e-3
    g = Grid(n, n, n, 2 * math.pi, 2 * math.pi, 2.0, beta=2.0)
    og = O.Grid(n, n, n, lx=g.lx, ly=g.ly, lz=2.0, beta=2.0)
    u, v, w = synth.uniform_velocity_np(2, n, n, n)
    pm = manufactured(g)
    gu, gv, gw = O.gradient(og, pm)
    us, vs, ws = u + dt * gu, v + dt * gv, w + dt * gw
    pg, po = check_against_oracle(g, prec, refine, us, vs, ws, dt=dt)
    pr, *_ = O.project(og, u, v, w, dt=dt)
    V = og.hz[:, None, None]
    pm0 = pm - np.sum(V * pm) / (np.sum(V) * n * n)
    assert rel_l2(pg - pr, pm0) <= 10 * TOL[prec]["phi"] * np.linalg.norm(po) / np.linalg.norm(pm0) + 1e-12


# ------------------------------------------------------------------ properties that hold at any size
def test_config2_full_size_properties():
    """256^3 (config 2 size), both precisions on the same inputs: the manufactured part of
    phi is recovered, the output is divergence-free, and FP64 and mixed agree."""
    n, dt = 256, 1e-3
    g = Grid(n, n, n, 2 * math.pi, 2 * math.pi, 2.0, beta=2.0)
    u, v, w = synth.uniform_velocity_torch(2, n, n, n, "cuda")
    res = {}
    for prec, refine in ((FP64, 0), (MIXED, 1)):
        plan = Plan([g], precision=prec, refine_steps=refine)
        (uo, vo, wo, po), st = plan.project(u, v, w, dt, stats=True)
        torch.cuda.synchronize()
        assert plan.sync_status() == 0
        res[prec] = po
        assert float(st["max_div"][0]) <= TOL[prec]["div"] * float(st["max_div_in"][0])
        plan.close()
    a, b = res[FP64], res[MIXED]
    assert float(torch.linalg.norm(a - b) / torch.linalg.norm(a)) <= 1e-9


# ------------------------------------------------------------------ in place, determinism, alpha dt
def test_in_place_and_deterministic():
    nx, ny, nz = 48, 32, 24
    g = Grid(nx, ny, nz, 1.0, 1.0, 1.0, beta=1.5)
    u, v, w = synth.uniform_velocity_np(5, nx, ny, nz)
    plan = Plan([g], precision=MIXED, refine_steps=1)
    a = plan.project(cuda(u), cuda(v), cuda(w), 1e-3)
    b = plan.project(cuda(u), cuda(v), cuda(w), 1e-3)
    for x, y in zip(a, b):
        assert torch.equal(x, y)
    ut, vt, wt = cuda(u), cuda(v), cuda(w)
    pt = torch.empty((nz, ny, nx), dtype=torch.float64, device="cuda")
    plan.project(ut, vt, wt, 1e-3, out=(ut, vt, wt, pt))
    for x, y in zip((ut, vt, wt, pt), a):
        assert torch.equal(x, y)


def test_alpha_dt_scaling():
    nx, ny, nz = 16, 16, 16
    g = Grid(nx, ny, nz, 1.0, 1.0, 1.0, beta=2.0)
    u, v, w = synth.uniform_velocity_np(6, nx, ny, nz)
    plan = Plan([g], precision=FP64)
    u1, v1, w1, p1 = plan.project(cuda(u), cuda(v), cuda(w), 1e-3, 1.0)
    for alpha in (8 / 15, 2 / 15, 1 / 3):   # the paper's RK3 alpha = gamma + rho
        u2, v2, w2, p2 = plan.project(cuda(u), cuda(v), cuda(w), 1e-3, alpha)
        assert float((u2 - u1).abs().max()) <= 1e-12
        assert float((p2 * alpha - p1).abs().max()) <= 1e-11 * float(p1.abs().max())


# ------------------------------------------------------------------ batch of uneven grids
def test_batch_uneven_grids_match_per_grid_oracle():
    draws = [(32, 24, 16, 1.3), (12, 48, 9, 2.7), (96, 64, 8, 1.0), (6, 6, 33, 2.0), (64, 32, 12, 2.5)]
    grids = [Grid(nx, ny, nz, 2 * math.pi, 2 * math.pi, 2.0, beta=b) for nx, ny, nz, b in draws]
    fields = [synth.uniform_velocity_np(1000 + i, *d[:3]) for i, d in enumerate(draws)]
    for prec in (FP64, MIXED):
        plan = Plan(grids, precision=prec, refine_steps=1 if prec == MIXED else 0)
        outs = plan.project_batch([tuple(cuda(a) for a in f) for f in fields], 1e-3)
        torch.cuda.synchronize()
        for g, f, o in zip(grids, fields, outs):
            og = O.Grid(g.nx, g.ny, g.nz, lx=g.lx, ly=g.ly, lz=g.lz, beta=g.beta)
            phi_o, uo, vo, wo, _ = O.project(og, *f)
            assert rel_l2(o[3].cpu().numpy(), phi_o) <= TOL[prec]["phi"]
            assert np.abs(o[0].cpu().numpy() - uo).max() <= TOL[prec]["u"]
        plan.close()


# ------------------------------------------------------------------ adjoint
@pytest.mark.parametrize("prec,tol", [(FP64, 1e-11), (MIXED, 1e-8)])
def test_adjoint_matches_oracle(prec, tol):
    nx, ny, nz = 16, 12, 10
    g = Grid(nx, ny, nz, 1.1, 0.9, 2.0, beta=2.0)
    og = O.Grid(nx, ny, nz, lx=1.1, ly=0.9, lz=2.0, beta=2.0)
    su, sv, sw = g.shapes
    gu, gv, gw = (synth.normal_np(6, i + 1, s) for i, s in enumerate((su, sv, sw)))
    gp = synth.normal_np(6, 4, (nz, ny, nx))
    ref = O.project_adjoint(og, gu, gv, gw, gp, dt=2e-3, alpha=0.5)
    plan = Plan([g], precision=prec, refine_steps=1 if prec == MIXED else 0)
    a, b, c = (torch.empty(s, dtype=torch.float64, device="cuda") for s in (su, sv, sw))
    plan.backward_into([(cuda(gu), cuda(gv), cuda(gw), cuda(gp))], [(a, b, c)], 2e-3, 0.5)
    torch.cuda.synchronize()
    for x, y in zip((a, b, c), ref):
        assert rel_l2(x.cpu().numpy(), y) <= tol


def test_autograd_function_dot_product():
    nx, ny, nz = 16, 16, 8
    g = Grid(nx, ny, nz, 1.0, 1.0, 1.0, beta=1.0)
    plan = Plan([g], precision=FP64)
    u, v, w = (cuda(a).requires_grad_(True) for a in synth.uniform_velocity_np(7, nx, ny, nz))
    wts = [cuda(synth.normal_np(8, i + 1, s)) for i, s in enumerate(g.shapes + ((nz, ny, nx),))]
    outs = Projection.apply(plan, 1e-3, 1.0, u, v, w)
    loss = sum((o * wt).sum() for o, wt in zip(outs, wts))
    loss.backward()
    lin = sum(float((gr * x).sum()) for gr, x in zip((u.grad, v.grad, w.grad), (u, v, w)))
    assert abs(lin - float(loss)) <= 1e-10 * (abs(float(loss)) + 1)

"""Homogeneous Dirichlet outlet for phi (bc_zhi = IBF_BC_DIRICHLET) on the GPU vs the oracle.

Section "Fluid Mechanics", boundary-condition paragraph: with neumann_velocity the
pressure-correction equation takes a homogeneous Dirichlet condition at the outlet.
phi = 0 on the top face (mirror value -phi_{nz-1}); the outlet face velocity is
corrected; no compatibility mean is removed and no reference value is fixed.
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
NEU, DIR = N.IBF_BC_NEUMANN, N.IBF_BC_DIRICHLET


@pytest.fixture(scope="module", autouse=True)
def _build():
    from paper_2609_19130_gb300 import build
    build.build()


def rel_l2(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def cuda(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to("cuda")


def make(nx, ny, nz, beta, wx=False, wy=False):
    g = Grid(nx, ny, nz, 2 * math.pi, 1.4, 2.0, beta=beta, bc_x=NEU if wx else 0, bc_y=NEU if wy else 0,
             bc_zhi=DIR)
    og = O.Grid(nx, ny, nz, lx=g.lx, ly=g.ly, lz=g.lz, beta=beta, wall_x=wx, wall_y=wy, dirichlet_top=True)
    return g, og


CASES = [(32, 24, 16, 2.0, False, False), (12, 6, 5, 1.0, False, False), (96, 64, 17, 2.5, False, False),
         (16, 12, 8, 1.5, True, True), (1, 1, 12, 2.0, False, False), (16, 16, 1, 0.0, False, False)]
VARIANTS = [None, dict(yz_kernel=2, mb=1, tri=1), dict(yz_kernel=2, mb=2, tri=2), dict(yz_kernel=3, mb=2)]


@pytest.mark.parametrize("case", CASES, ids=lambda c: "{}x{}x{}{}".format(*c[:3], "_walls" if c[4] else ""))
@pytest.mark.parametrize("prec", [FP64, MIXED])
def test_outlet_matches_oracle(case, prec):
    nx, ny, nz, beta, wx, wy = case
    g, og = make(nx, ny, nz, beta, wx, wy)
    # outflow through the outlet that does not balance the inflow: nothing is removed
    u, v, w = synth.uniform_velocity_np(61, nx, ny, nz, wall_x=wx, wall_y=wy)
    w[-1] = synth.uniform_np(62, 1, w[-1].shape, 0.0, 1.0)
    phi_o, u_o, v_o, w_o, st_o = O.project(og, u, v, w, dt=2e-3, alpha=0.5)
    umax = max(np.abs(u).max(), np.abs(v).max(), np.abs(w).max())
    t = TOL[prec]
    for var in VARIANTS:
        if var and var.get("tri", 0) > 1 + int(math.floor(math.log2(nz))):
            continue
        plan = Plan([g], precision=prec, refine_steps=1 if prec == MIXED else 0,
                    tuning=[var] if var else None)
        (uo, vo, wo, po), st = plan.project(cuda(u), cuda(v), cuda(w), 2e-3, 0.5, stats=True)
        torch.cuda.synchronize()
        assert plan.sync_status() == 0          # no incompatibility warning with an outlet
        plan.close()
        pg = po.cpu().numpy()
        assert rel_l2(pg, phi_o) <= t["phi"], (var, rel_l2(pg, phi_o))
        for a, b in ((uo, u_o), (vo, v_o), (wo, w_o)):
            assert np.abs(a.cpu().numpy() - b).max() <= t["u"] * umax, (var, np.abs(a.cpu().numpy() - b).max())
        assert np.array_equal(wo.cpu().numpy()[0], w[0])     # bottom wall untouched
        assert float(st["compat"][0]) == 0.0
        assert float(st["max_div"][0]) <= t["div"] * st_o[1]


@pytest.mark.parametrize("prec,tol", [(FP64, 1e-11), (MIXED, 1e-8)])
def test_outlet_adjoint_matches_oracle(prec, tol):
    nx, ny, nz = 16, 12, 10
    g, og = make(nx, ny, nz, 2.0)
    su, sv, sw = g.shapes
    gu, gv, gw = (synth.normal_np(63, i + 1, s) for i, s in enumerate((su, sv, sw)))
    gp = synth.normal_np(63, 4, (nz, ny, nx))
    ref = O.project_adjoint(og, gu, gv, gw, gp, dt=2e-3, alpha=0.5)
    plan = Plan([g], precision=prec, refine_steps=1 if prec == MIXED else 0)
    a, b, c = (torch.empty(s, dtype=torch.float64, device="cuda") for s in (su, sv, sw))
    plan.backward_into([(cuda(gu), cuda(gv), cuda(gw), cuda(gp))], [(a, b, c)], 2e-3, 0.5)
    torch.cuda.synchronize()
    plan.close()
    for x, y in zip((a, b, c), ref):
        assert rel_l2(x.cpu().numpy(), y) <= tol, rel_l2(x.cpu().numpy(), y)


def test_batch_mixing_outlet_and_walls():
    """One plan over grids with a Neumann top and with a Dirichlet outlet."""
    specs = [(32, 24, 16, 1.3, NEU), (24, 16, 12, 2.0, DIR), (16, 16, 9, 1.0, DIR)]
    grids = [Grid(nx, ny, nz, 2 * math.pi, 2 * math.pi, 2.0, beta=b, bc_zhi=top) for nx, ny, nz, b, top in specs]
    fields = [synth.uniform_velocity_np(70 + i, *s[:3]) for i, s in enumerate(specs)]
    for prec in (FP64, MIXED):
        plan = Plan(grids, precision=prec, refine_steps=1 if prec == MIXED else 0)
        outs = plan.project_batch([tuple(cuda(a) for a in f) for f in fields], 1e-3)
        torch.cuda.synchronize()
        for gr, f, o in zip(grids, fields, outs):
            og = O.Grid(gr.nx, gr.ny, gr.nz, lx=gr.lx, ly=gr.ly, lz=gr.lz, beta=gr.beta,
                        dirichlet_top=gr.bc_zhi == DIR)
            phi_o, uo, vo, wo, _ = O.project(og, *f)
            assert rel_l2(o[3].cpu().numpy(), phi_o) <= TOL[prec]["phi"]
            assert np.abs(o[2].cpu().numpy() - wo).max() <= TOL[prec]["u"]
        plan.close()
